// Host-side planner: operator algebra, term generation, compression.
// See plan.hpp for the paper references.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <iterator>
#include <limits>
#include <sstream>
#include <stdexcept>
#include <unordered_map>
#include <utility>

namespace dmrg {

// ---------------------------------------------------------------- 4x4 algebra

Mat4 mat_zero() { Mat4 m; m.fill(0.0); return m; }
Mat4 mat_eye() { Mat4 m = mat_zero(); for (int i = 0; i < 4; ++i) m[i * 5] = 1.0; return m; }
Mat4 mat_mul(const Mat4 &a, const Mat4 &b) {
  Mat4 c = mat_zero();
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      const double x = a[i * 4 + k];
      if (x == 0.0) continue;
      for (int j = 0; j < 4; ++j) c[i * 4 + j] += x * b[k * 4 + j];
    }
  return c;
}
Mat4 mat_t(const Mat4 &a) {
  Mat4 c;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) c[i * 4 + j] = a[j * 4 + i];
  return c;
}
Mat4 mat_scale(const Mat4 &a, double s) { Mat4 c = a; for (auto &x : c) x *= s; return c; }
static Mat4 mat_add(const Mat4 &a, const Mat4 &b) { Mat4 c = a; for (int i = 0; i < 16; ++i) c[i] += b[i]; return c; }
bool mat_is_zero(const Mat4 &a) { for (double x : a) if (x != 0.0) return false; return true; }
int mat_parity(const Mat4 &a) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c)
      if (a[r * 4 + c] != 0.0) return (SITE_NU[r] + SITE_ND[r] + SITE_NU[c] + SITE_ND[c]) & 1;
  return 0;
}

// Eq. creation_ops in the basis {0, up, dn, updn} with |updn> = a+_up a+_dn |0>.
static Mat4 site_cdag_spin(int spin) {
  Mat4 m = mat_zero();
  if (spin == 0) { m[1 * 4 + 0] = 1.0; m[3 * 4 + 2] = 1.0; }
  else { m[2 * 4 + 0] = 1.0; m[3 * 4 + 1] = -1.0; }
  return m;
}

Mat4 SiteAlgebra::cdag(int p) const { return site_cdag_spin(p & 1); }
Mat4 SiteAlgebra::c(int p) const { return mat_t(site_cdag_spin(p & 1)); }

Mat4 SiteAlgebra::H(int s) const {
  Mat4 m = mat_zero();
  const int md[2] = {2 * s, 2 * s + 1};
  for (int p : md)
    for (int q : md)
      if (I->t(p, q) != 0.0) m = mat_add(m, mat_scale(mat_mul(cdag(p), c(q)), I->t(p, q)));
  for (int p : md) for (int q : md) for (int r : md) for (int t : md) {
    const double x = I->w(p, q, r, t);
    if (x == 0.0 || p == q || r == t) continue;
    m = mat_add(m, mat_scale(mat_mul(mat_mul(cdag(p), cdag(q)), mat_mul(c(t), c(r))), 0.5 * x));
  }
  return m;
}

Mat4 SiteAlgebra::T(int s, int j) const {
  Mat4 m = mat_zero();
  const int md[2] = {2 * s, 2 * s + 1};
  for (int i : md)
    if (I->t(i, j) != 0.0) m = mat_add(m, mat_scale(cdag(i), I->t(i, j)));
  for (int p : md) for (int q : md) for (int r : md) {
    const double x = I->w(p, q, r, j);
    if (x == 0.0 || p == q) continue;
    m = mat_add(m, mat_scale(mat_mul(mat_mul(cdag(p), cdag(q)), c(r)), -x));
  }
  return m;
}

Mat4 SiteAlgebra::V(int s, int i) const {
  Mat4 m = mat_zero();
  const int md[2] = {2 * s, 2 * s + 1};
  for (int q : md) for (int r : md) for (int t : md) {
    const double x = I->w(i, q, r, t);
    if (x == 0.0 || r == t) continue;
    m = mat_add(m, mat_scale(mat_mul(mat_mul(cdag(q), c(t)), c(r)), x));
  }
  return m;
}

Mat4 SiteAlgebra::Pc(int s, int r, int q) const {
  const int a = 2 * s, b = 2 * s + 1;
  return mat_scale(mat_mul(cdag(a), cdag(b)), I->W(a, b, r, q));
}

Mat4 SiteAlgebra::Pa(int s, int p, int q) const {
  const int a = 2 * s, b = 2 * s + 1;
  return mat_scale(mat_mul(c(b), c(a)), I->W(p, q, a, b));
}

Mat4 SiteAlgebra::Q(int s, int p, int q) const {
  Mat4 m = mat_zero();
  const int md[2] = {2 * s, 2 * s + 1};
  for (int a : md) for (int b : md) {
    const double x = I->w(p, a, q, b) - I->w(p, a, b, q);
    if (x != 0.0) m = mat_add(m, mat_scale(mat_mul(cdag(a), c(b)), x));
  }
  return m;
}

// ---------------------------------------------------------------- layouts

int BlockLayout::find(int nu, int nd) const {
  int lo = 0, hi = (int)sec.size() - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) / 2;
    const Sector &s = sec[mid];
    if (s.nu == nu && s.nd == nd) return mid;
    if (s.nu < nu || (s.nu == nu && s.nd < nd)) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

bool BlockLayout::has_site(int s) const {
  return std::binary_search(sites.begin(), sites.end(), s);
}

bool BlockLayout::get(int kind, int i, int j, int &f, int &k) const {
  auto it = lookup.find(key(kind, i, j, L));
  if (it == lookup.end()) return false;
  f = it->second.first;
  k = it->second.second;
  return true;
}

static void dq_of(int kind, int i, int j, int &du, int &dd) {
  auto e = [](int p, int &u, int &d, int sgn) { if ((p & 1) == 0) u += sgn; else d += sgn; };
  du = dd = 0;
  switch (kind) {
    case KH: break;
    case KC: case KT: e(i, du, dd, +1); break;
    case KV: e(i, du, dd, -1); break;
    case KA: e(i, du, dd, +1); e(j, du, dd, +1); break;
    case KB: e(i, du, dd, +1); e(j, du, dd, -1); break;
  }
}

void build_layout(BlockLayout &b, int side, int L, const std::vector<int> &sites,
                  const std::vector<Sector> &sec) {
  b.side = side;
  b.L = L;
  b.sites = sites;
  b.sec = sec;
  b.fam.clear();
  b.lookup.clear();
  if (sites.empty()) { b.total = 0; return; }
  std::vector<int> modes;
  for (int s : sites) { modes.push_back(2 * s); modes.push_back(2 * s + 1); }
  auto add_family = [&](int kind, const std::vector<std::array<int, 2>> &idx) {
    if (idx.empty()) return;
    // split by quantum-number change
    std::map<std::pair<int, int>, std::vector<std::array<int, 2>>> groups;
    for (auto &ij : idx) {
      int du, dd;
      dq_of(kind, ij[0], ij[1], du, dd);
      groups[{du, dd}].push_back(ij);
    }
    for (auto &g : groups) {
      Family f;
      f.kind = kind;
      f.dnu = g.first.first;
      f.dnd = g.first.second;
      f.idx = g.second;
      b.fam.push_back(f);
    }
  };
  add_family(KH, {{-1, -1}});
  {
    std::vector<std::array<int, 2>> v;
    for (int p : modes) v.push_back({p, -1});
    add_family(KC, v);
  }
  if (side == 0) {
    std::vector<std::array<int, 2>> v;
    for (int s = sites.back() + 1; s < L; ++s) { v.push_back({2 * s, -1}); v.push_back({2 * s + 1, -1}); }
    add_family(KT, v);
  } else {
    std::vector<std::array<int, 2>> v;
    for (int s = 0; s < sites.front(); ++s) { v.push_back({2 * s, -1}); v.push_back({2 * s + 1, -1}); }
    add_family(KV, v);
  }
  {
    std::vector<std::array<int, 2>> va, vb;
    for (int p : modes)
      for (int q : modes) {
        if (p < q) va.push_back({p, q});
        vb.push_back({p, q});
      }
    add_family(KA, va);
    add_family(KB, vb);
  }
  int64_t cur = 0;
  for (int fi = 0; fi < (int)b.fam.size(); ++fi) {
    Family &f = b.fam[fi];
    f.base = cur;
    f.bra.assign(sec.size(), -1);
    f.off.assign(sec.size(), -1);
    int64_t o = 0;
    for (int a = 0; a < (int)sec.size(); ++a) {
      const int br = b.find(sec[a].nu + f.dnu, sec[a].nd + f.dnd);
      f.bra[a] = br;
      if (br < 0) continue;
      f.off[a] = o;
      o += (int64_t)f.K() * sec[br].dim * sec[a].dim;
    }
    f.size = o;
    cur += o;
    for (int k = 0; k < f.K(); ++k)
      b.lookup[BlockLayout::key(f.kind, f.idx[k][0], f.idx[k][1], L)] = {fi, k};
  }
  b.total = cur;
}

// ---------------------------------------------------------------- op refs

int OpRef::parity() const {
  if (type == 0) return 0;
  switch (kind) {
    case KC: case KT: case KV: return 1;
    default: return 0;
  }
}

static OpRef ident() { return OpRef(); }
static OpRef stored(int kind, int i, int j = -1, bool tr = false) {
  OpRef o; o.type = 1; o.kind = kind; o.i = i; o.j = j; o.tr = tr; return o;
}
static OpRef lincomb(int kind, bool tr, const std::vector<std::tuple<int, int, double>> &lc) {
  OpRef o; o.type = 2; o.kind = kind; o.tr = tr;
  for (auto &x : lc) if (std::get<2>(x) != 0.0) o.lc.push_back(x);
  return o;
}

// ---------------------------------------------------------------- half operators

HalfOps::HalfOps(const Integrals *I_, int k_, bool le, bool re)
    : I(I_), L(I_->L), k(k_), lsites(k_), rfirst(k_ + 2), S{I_}, l_empty(le), r_empty(re) {}

static void push(HalfOp &h, const OpRef &o, const Mat4 &s, double c) {
  if (c == 0.0 || mat_is_zero(s)) return;
  if (o.type == 2 && o.lc.empty()) return;
  h.push_back({o, s, c});
}

// sum_u X_u (x) S_u  ->  sum_E (sum_u S_u[E] X_u) (x) E for block ops of one kind
static void sum_over(HalfOp &h, int kind, bool tr,
                     const std::vector<std::tuple<int, int, Mat4, double>> &terms) {
  for (int e = 0; e < 16; ++e) {
    std::vector<std::tuple<int, int, double>> lc;
    for (auto &t : terms) {
      const double x = std::get<2>(t)[e] * std::get<3>(t);
      if (x != 0.0) lc.emplace_back(std::get<0>(t), std::get<1>(t), x);
    }
    if (lc.empty()) continue;
    Mat4 E = mat_zero();
    E[e] = 1.0;
    push(h, lincomb(kind, tr, lc), E, 1.0);
  }
}

HalfOp HalfOps::L_I() const { return {{ident(), mat_eye(), 1.0}}; }

HalfOp HalfOps::L_C(int p) const {
  HalfOp h;
  if (in_l(p)) push(h, stored(KC, p), mat_eye(), 1.0);
  else push(h, ident(), S.cdag(p), 1.0);
  return h;
}

HalfOp HalfOps::L_A(int p, int q) const {
  HalfOp h;
  if (in_l(p) && in_l(q)) push(h, stored(KA, p, q), mat_eye(), 1.0);
  else if (in_l(p)) push(h, stored(KC, p), S.cdag(q), 1.0);
  else push(h, ident(), mat_mul(S.cdag(p), S.cdag(q)), 1.0);
  return h;
}

HalfOp HalfOps::L_B(int p, int s) const {
  HalfOp h;
  if (in_l(p) && in_l(s)) push(h, stored(KB, p, s), mat_eye(), 1.0);
  else if (in_l(p)) push(h, stored(KC, p), S.c(s), 1.0);
  else if (in_l(s)) push(h, stored(KC, s, -1, true), S.cdag(p), -1.0);
  else push(h, ident(), mat_mul(S.cdag(p), S.c(s)), 1.0);
  return h;
}

HalfOp HalfOps::L_H() const {
  HalfOp h;
  const int sl[2] = {2 * k, 2 * k + 1};
  push(h, stored(KH, -1), mat_eye(), 1.0);
  push(h, ident(), S.H(k), 1.0);
  for (int j : sl) {  // T^l_j c_j + h.c.
    push(h, stored(KT, j), S.c(j), 1.0);
    push(h, stored(KT, j, -1, true), S.cdag(j), -1.0);
  }
  {  // c+_i V^sl_i + h.c.
    std::vector<std::tuple<int, int, Mat4, double>> a, b;
    for (int i = 0; i < 2 * k; ++i) {
      const Mat4 v = S.V(k, i);
      a.emplace_back(i, -1, v, 1.0);
      b.emplace_back(i, -1, mat_t(v), -1.0);
    }
    sum_over(h, KC, false, a);
    sum_over(h, KC, true, b);
  }
  {  // Pc^l_{rs} (c_s c_r)^sl + h.c.
    const int r = sl[0], s = sl[1];
    std::vector<std::tuple<int, int, double>> lc;
    for (int p = 0; p < 2 * k; ++p)
      for (int q = p + 1; q < 2 * k; ++q) lc.emplace_back(p, q, I->W(p, q, r, s));
    const Mat4 cc = mat_mul(S.c(s), S.c(r));
    push(h, lincomb(KA, false, lc), cc, 1.0);
    push(h, lincomb(KA, true, lc), mat_t(cc), 1.0);
  }
  for (int a : sl)  // Q^l_{ab} (c+_a c_b)^sl
    for (int b : sl) {
      std::vector<std::tuple<int, int, double>> lc;
      for (int q = 0; q < 2 * k; ++q)
        for (int r = 0; r < 2 * k; ++r) lc.emplace_back(q, r, I->w(a, q, b, r) - I->w(a, q, r, b));
      push(h, lincomb(KB, false, lc), mat_mul(S.cdag(a), S.c(b)), 1.0);
    }
  return h;
}

HalfOp HalfOps::L_T(int j) const {
  HalfOp h;
  const int sl[2] = {2 * k, 2 * k + 1};
  push(h, stored(KT, j), mat_eye(), 1.0);
  push(h, ident(), S.T(k, j), 1.0);
  for (int r : sl) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int p = 0; p < 2 * k; ++p)
      for (int q = p + 1; q < 2 * k; ++q) lc.emplace_back(p, q, I->W(p, q, r, j));
    push(h, lincomb(KA, false, lc), S.c(r), -1.0);
  }
  for (int q : sl) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int a = 0; a < 2 * k; ++a)
      for (int b = 0; b < 2 * k; ++b) lc.emplace_back(a, b, I->w(q, a, j, b) - I->w(q, a, b, j));
    push(h, lincomb(KB, false, lc), S.cdag(q), 1.0);
  }
  {
    std::vector<std::tuple<int, int, Mat4, double>> a, b;
    for (int p = 0; p < 2 * k; ++p) {
      a.emplace_back(p, -1, S.Q(k, p, j), 1.0);
      b.emplace_back(p, -1, S.Pc(k, p, j), -1.0);
    }
    sum_over(h, KC, false, a);
    sum_over(h, KC, true, b);
  }
  return h;
}

HalfOp HalfOps::L_Pc(int r, int s) const {
  HalfOp h;
  const int sl[2] = {2 * k, 2 * k + 1};
  {
    std::vector<std::tuple<int, int, double>> lc;
    for (int p = 0; p < 2 * k; ++p)
      for (int q = p + 1; q < 2 * k; ++q) lc.emplace_back(p, q, I->W(p, q, r, s));
    push(h, lincomb(KA, false, lc), mat_eye(), 1.0);
  }
  push(h, ident(), S.Pc(k, r, s), 1.0);
  for (int q : sl) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int p = 0; p < 2 * k; ++p) lc.emplace_back(p, -1, I->W(p, q, r, s));
    push(h, lincomb(KC, false, lc), S.cdag(q), 1.0);
  }
  return h;
}

HalfOp HalfOps::L_Q(int a, int b) const {
  HalfOp h;
  const int sl[2] = {2 * k, 2 * k + 1};
  auto coef = [&](int q, int r) { return I->w(a, q, b, r) - I->w(a, q, r, b); };
  {
    std::vector<std::tuple<int, int, double>> lc;
    for (int q = 0; q < 2 * k; ++q)
      for (int r = 0; r < 2 * k; ++r) lc.emplace_back(q, r, coef(q, r));
    push(h, lincomb(KB, false, lc), mat_eye(), 1.0);
  }
  push(h, ident(), S.Q(k, a, b), 1.0);
  for (int r : sl) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int q = 0; q < 2 * k; ++q) lc.emplace_back(q, -1, coef(q, r));
    push(h, lincomb(KC, false, lc), S.c(r), 1.0);
  }
  for (int q : sl) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int r = 0; r < 2 * k; ++r) lc.emplace_back(r, -1, coef(q, r));
    push(h, lincomb(KC, true, lc), S.cdag(q), -1.0);
  }
  return h;
}

HalfOp HalfOps::R_I() const { return {{ident(), mat_eye(), 1.0}}; }

HalfOp HalfOps::R_C(int p) const {
  HalfOp h;
  if (is_sr(p)) push(h, ident(), S.cdag(p), 1.0);
  else push(h, stored(KC, p), mat_eye(), 1.0);
  return h;
}

HalfOp HalfOps::R_c(int p) const {
  HalfOp h;
  if (is_sr(p)) push(h, ident(), S.c(p), 1.0);
  else push(h, stored(KC, p, -1, true), mat_eye(), 1.0);
  return h;
}

HalfOp HalfOps::R_A(int p, int q) const {
  HalfOp h;
  if (is_sr(p) && is_sr(q)) push(h, ident(), mat_mul(S.cdag(p), S.cdag(q)), 1.0);
  else if (is_sr(p)) push(h, stored(KC, q), S.cdag(p), 1.0);
  else push(h, stored(KA, p, q), mat_eye(), 1.0);
  return h;
}

HalfOp HalfOps::R_AT(int p, int q) const {
  HalfOp h;
  if (is_sr(p) && is_sr(q)) push(h, ident(), mat_t(mat_mul(S.cdag(p), S.cdag(q))), 1.0);
  else if (is_sr(p)) push(h, stored(KC, q, -1, true), S.c(p), -1.0);
  else push(h, stored(KA, p, q, true), mat_eye(), 1.0);
  return h;
}

HalfOp HalfOps::R_B(int p, int s) const {
  HalfOp h;
  if (is_sr(p) && is_sr(s)) push(h, ident(), mat_mul(S.cdag(p), S.c(s)), 1.0);
  else if (is_sr(p)) push(h, stored(KC, s, -1, true), S.cdag(p), 1.0);
  else if (is_sr(s)) push(h, stored(KC, p), S.c(s), -1.0);
  else push(h, stored(KB, p, s), mat_eye(), 1.0);
  return h;
}

HalfOp HalfOps::R_H() const {
  HalfOp h;
  const int s1 = k + 1;
  const int sr[2] = {2 * s1, 2 * s1 + 1};
  push(h, stored(KH, -1), mat_eye(), 1.0);
  push(h, ident(), S.H(s1), 1.0);
  {  // T^sr_j c_j + h.c., j in r
    std::vector<std::tuple<int, int, Mat4, double>> a, b;
    for (int j = 2 * (k + 2); j < 2 * L; ++j) {
      const Mat4 t = S.T(s1, j);
      a.emplace_back(j, -1, t, 1.0);
      b.emplace_back(j, -1, mat_t(t), -1.0);
    }
    sum_over(h, KC, true, a);
    sum_over(h, KC, false, b);
  }
  for (int i : sr) {  // c+_i V^r_i + h.c.
    push(h, stored(KV, i), S.cdag(i), 1.0);
    push(h, stored(KV, i, -1, true), S.c(i), -1.0);
  }
  {  // A^sr_pq Pa^r_pq + h.c.
    const int p = sr[0], q = sr[1];
    std::vector<std::tuple<int, int, double>> lc;
    for (int r = 2 * (k + 2); r < 2 * L; ++r)
      for (int s = r + 1; s < 2 * L; ++s) lc.emplace_back(r, s, I->W(p, q, r, s));
    const Mat4 aa = mat_mul(S.cdag(p), S.cdag(q));
    push(h, lincomb(KA, true, lc), aa, 1.0);
    push(h, lincomb(KA, false, lc), mat_t(aa), 1.0);
  }
  for (int p : sr)  // B^sr_ps Q^r_ps
    for (int s : sr) {
      std::vector<std::tuple<int, int, double>> lc;
      for (int q = 2 * (k + 2); q < 2 * L; ++q)
        for (int r = 2 * (k + 2); r < 2 * L; ++r) lc.emplace_back(q, r, I->w(p, q, s, r) - I->w(p, q, r, s));
      push(h, lincomb(KB, false, lc), mat_mul(S.cdag(p), S.c(s)), 1.0);
    }
  return h;
}

HalfOp HalfOps::R_V(int i) const {
  HalfOp h;
  const int s1 = k + 1;
  const int sr[2] = {2 * s1, 2 * s1 + 1};
  const int r0 = 2 * (k + 2);
  push(h, ident(), S.V(s1, i), 1.0);
  push(h, stored(KV, i), mat_eye(), 1.0);
  for (int q : sr) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int r = r0; r < 2 * L; ++r)
      for (int s = r + 1; s < 2 * L; ++s) lc.emplace_back(r, s, I->W(i, q, r, s));
    push(h, lincomb(KA, true, lc), S.cdag(q), 1.0);
  }
  {
    std::vector<std::tuple<int, int, Mat4, double>> a;
    for (int q = r0; q < 2 * L; ++q) a.emplace_back(q, -1, S.Pa(s1, i, q), 1.0);
    sum_over(h, KC, false, a);
  }
  for (int q : sr)
    for (int s : sr) {
      std::vector<std::tuple<int, int, double>> lc;
      for (int r = r0; r < 2 * L; ++r) lc.emplace_back(r, -1, I->w(i, q, r, s) - I->w(i, q, s, r));
      push(h, lincomb(KC, true, lc), mat_mul(S.cdag(q), S.c(s)), 1.0);
    }
  for (int s : sr) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int q = r0; q < 2 * L; ++q)
      for (int r = r0; r < 2 * L; ++r) lc.emplace_back(q, r, I->w(i, q, s, r) - I->w(i, q, r, s));
    push(h, lincomb(KB, false, lc), S.c(s), 1.0);
  }
  return h;
}

HalfOp HalfOps::R_Pa(int p, int q) const {
  HalfOp h;
  const int s1 = k + 1;
  const int sr[2] = {2 * s1, 2 * s1 + 1};
  const int r0 = 2 * (k + 2);
  push(h, ident(), S.Pa(s1, p, q), 1.0);
  {
    std::vector<std::tuple<int, int, double>> lc;
    for (int r = r0; r < 2 * L; ++r)
      for (int s = r + 1; s < 2 * L; ++s) lc.emplace_back(r, s, I->W(p, q, r, s));
    push(h, lincomb(KA, true, lc), mat_eye(), 1.0);
  }
  for (int r : sr) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int s = r0; s < 2 * L; ++s) lc.emplace_back(s, -1, I->W(p, q, r, s));
    push(h, lincomb(KC, true, lc), S.c(r), -1.0);
  }
  return h;
}

HalfOp HalfOps::R_Q(int a, int b) const {
  HalfOp h;
  const int s1 = k + 1;
  const int sr[2] = {2 * s1, 2 * s1 + 1};
  const int r0 = 2 * (k + 2);
  auto coef = [&](int q, int r) { return I->w(a, q, b, r) - I->w(a, q, r, b); };
  push(h, ident(), S.Q(s1, a, b), 1.0);
  {
    std::vector<std::tuple<int, int, double>> lc;
    for (int q = r0; q < 2 * L; ++q)
      for (int r = r0; r < 2 * L; ++r) lc.emplace_back(q, r, coef(q, r));
    push(h, lincomb(KB, false, lc), mat_eye(), 1.0);
  }
  for (int q : sr) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int r = r0; r < 2 * L; ++r) lc.emplace_back(r, -1, coef(q, r));
    push(h, lincomb(KC, true, lc), S.cdag(q), 1.0);
  }
  for (int r : sr) {
    std::vector<std::tuple<int, int, double>> lc;
    for (int q = r0; q < 2 * L; ++q) lc.emplace_back(q, -1, coef(q, r));
    push(h, lincomb(KC, false, lc), S.c(r), -1.0);
  }
  return h;
}

// ---------------------------------------------------------------- H terms

static void product(std::vector<Piece> &out, const HalfOp &l, const HalfOp &r, double c, bool hc) {
  for (auto &a : l)
    for (auto &b : r) {
      const double x = a.coef * b.coef * c;
      if (x == 0.0) continue;
      out.push_back({x, a.blk, a.site, b.site, b.blk, hc});
    }
}

std::vector<Piece> hamiltonian_pieces(const Integrals &I, int k, bool l_empty, bool r_empty) {
  HalfOps O(&I, k, l_empty, r_empty);
  const int L = I.L;
  std::vector<Piece> ps;
  product(ps, O.L_H(), O.R_I(), 1.0, false);
  product(ps, O.L_I(), O.R_H(), 1.0, false);
  const int lp_end = 2 * (k + 1);  // L' modes [0, lp_end), R' modes [lp_end, 2L)
  for (int j = lp_end; j < 2 * L; ++j) product(ps, O.L_T(j), O.R_c(j), 1.0, true);
  for (int i = 0; i < lp_end; ++i) product(ps, O.L_C(i), O.R_V(i), 1.0, true);
  const bool normal_on_left = (k + 1) <= (L - k - 1);
  // the pair terms, one row of pair indices per task, appended in row order
  auto rows = [&](int lo, int hi, auto &&row) {
    std::vector<std::vector<Piece>> part((size_t)(hi - lo));
    parallel_for(part.size(), [&](size_t i) { row((int)i + lo, part[i]); });
    for (auto &v : part) ps.insert(ps.end(), std::make_move_iterator(v.begin()), std::make_move_iterator(v.end()));
  };
  if (normal_on_left) {
    rows(0, lp_end, [&](int p, std::vector<Piece> &out) {
      for (int q = p + 1; q < lp_end; ++q) product(out, O.L_A(p, q), O.R_Pa(p, q), 1.0, true);
    });
    rows(0, lp_end, [&](int p, std::vector<Piece> &out) {
      for (int s = 0; s < lp_end; ++s) product(out, O.L_B(p, s), O.R_Q(p, s), 1.0, false);
    });
  } else {
    rows(lp_end, 2 * L, [&](int r, std::vector<Piece> &out) {
      for (int s = r + 1; s < 2 * L; ++s) product(out, O.L_Pc(r, s), O.R_AT(r, s), 1.0, true);
    });
    rows(lp_end, 2 * L, [&](int q, std::vector<Piece> &out) {
      for (int r = lp_end; r < 2 * L; ++r) product(out, O.L_Q(q, r), O.R_B(q, r), 1.0, false);
    });
  }
  // drop pieces on operators of empty blocks (all zero there)
  std::vector<Piece> out;
  for (auto &p : ps) {
    if (l_empty && p.l.type != 0) continue;
    if (r_empty && p.r.type != 0) continue;
    out.push_back(std::move(p));
  }
  return out;
}

// ---------------------------------------------------------------- compression

// Exact identity of an operator reference (coefficients compared bit for bit).
static bool same_op(const OpRef &a, const OpRef &b) {
  if (a.type != b.type || a.kind != b.kind || a.i != b.i || a.j != b.j || a.tr != b.tr) return false;
  if (a.type != 2) return true;
  if (a.lc.size() != b.lc.size()) return false;
  for (size_t t = 0; t < a.lc.size(); ++t) {
    if (std::get<0>(a.lc[t]) != std::get<0>(b.lc[t]) || std::get<1>(a.lc[t]) != std::get<1>(b.lc[t])) return false;
    uint64_t x, y;
    const double cx = std::get<2>(a.lc[t]), cy = std::get<2>(b.lc[t]);
    std::memcpy(&x, &cx, 8);
    std::memcpy(&y, &cy, 8);
    if (x != y) return false;
  }
  return true;
}

static uint64_t mix(uint64_t h, uint64_t x) {
  h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

static uint64_t op_hash(const OpRef &o) {
  uint64_t h = mix(mix(mix(mix(mix(0, (uint64_t)o.type), (uint64_t)(o.kind + 1)), (uint64_t)(o.i + 1)),
                       (uint64_t)(o.j + 1)), (uint64_t)o.tr);
  if (o.type == 2)
    for (const auto &t : o.lc) {
      uint64_t bits;
      const double c = std::get<2>(t);
      std::memcpy(&bits, &c, 8);
      h = mix(mix(mix(h, (uint64_t)std::get<0>(t)), (uint64_t)std::get<1>(t)), bits);
    }
  return h;
}

// The pieces that can be merged: same exact operator on the fixed side, same
// family (kind, transpose, quantum-number change) on the varying side, same
// Hermitian-conjugate flag.
struct MergeKey {
  const OpRef *fixed;
  int kind, du, dd;
  bool tr, hc;
  uint64_t hash;
};
struct MergeKeyHash {
  size_t operator()(const MergeKey &k) const { return (size_t)k.hash; }
};
struct MergeKeyEq {
  bool operator()(const MergeKey &a, const MergeKey &b) const {
    return a.hash == b.hash && a.kind == b.kind && a.du == b.du && a.dd == b.dd && a.tr == b.tr &&
           a.hc == b.hc && same_op(*a.fixed, *b.fixed);
  }
};

// side 0: merge the left operators of pieces sharing the exact right operator.
static std::vector<Piece> compress_side(std::vector<Piece> in, int side) {
  std::unordered_map<MergeKey, int, MergeKeyHash, MergeKeyEq> index;
  std::vector<std::vector<int>> groups;  // in order of first appearance
  for (int i = 0; i < (int)in.size(); ++i) {
    const Piece &p = in[i];
    const OpRef &fixed = side == 0 ? p.r : p.l;
    const OpRef &var = side == 0 ? p.l : p.r;
    if (var.type == 0) {  // identity on the varying side: nothing to merge
      groups.push_back({i});
      continue;
    }
    int vi = var.i, vj = var.j;
    if (var.type == 2) {
      vi = std::get<0>(var.lc[0]);
      vj = std::get<1>(var.lc[0]);
    }
    MergeKey k{&fixed, var.kind, 0, 0, var.tr, p.hc, 0};
    dq_of(var.kind, vi, vj, k.du, k.dd);
    k.hash = mix(mix(mix(mix(mix(op_hash(fixed), (uint64_t)(var.kind + 1)), (uint64_t)var.tr),
                         (uint64_t)(k.du + 64)), (uint64_t)(k.dd + 64)), (uint64_t)p.hc);
    auto it = index.find(k);
    if (it == index.end()) {
      index.emplace(k, (int)groups.size());
      groups.push_back({i});
    } else {
      groups[it->second].push_back(i);
    }
  }
  // Merged sources per elementary site pair, accumulated in dense arrays over
  // the source index (i + 1, j + 1): every source receives its contributions
  // in the order of the pieces, and both the site pairs and the sources come
  // out in ascending order.  Groups are independent: chunks of them run in
  // parallel, each thread reusing its own buffers, and the outputs are joined
  // in group order.
  const size_t CD = 256;
  std::vector<int> dmax((in.size() + CD - 1) / CD, 2);
  parallel_for(dmax.size(), [&](size_t ch) {
    int m = 2;
    for (size_t i = ch * CD; i < std::min(in.size(), (ch + 1) * CD); ++i)
      for (const OpRef *o : {&in[i].l, &in[i].r}) {
        m = std::max(m, std::max(o->i, o->j) + 2);
        for (const auto &t : o->lc) m = std::max(m, std::max(std::get<0>(t), std::get<1>(t)) + 2);
      }
    dmax[ch] = m;
  });
  int D = 2;
  for (int m : dmax) D = std::max(D, m);
  struct Acc {
    std::vector<double> val;
    std::vector<char> used;
    std::vector<int> touched;
  };
  std::vector<std::vector<Piece>> gout(groups.size());
  const size_t CH = 64;
  parallel_for((groups.size() + CH - 1) / CH, [&](size_t ch) {
    thread_local std::vector<Acc> pool;
    thread_local std::vector<int> slot_of, pairs;
    if (slot_of.size() != 256) slot_of.assign(256, -1);
    for (size_t gi = ch * CH; gi < std::min(groups.size(), (ch + 1) * CH); ++gi) {
      const std::vector<int> &g = groups[gi];
      if (g.size() == 1) {
        gout[gi].push_back(std::move(in[(size_t)g[0]]));
        continue;
      }
      pairs.clear();
      for (int i : g) {
        const Piece &p = in[(size_t)i];
        const OpRef &var = side == 0 ? p.l : p.r;
        for (int e1 = 0; e1 < 16; ++e1) {
          if (p.sl[e1] == 0.0) continue;
          for (int e2 = 0; e2 < 16; ++e2) {
            if (p.sr[e2] == 0.0) continue;
            const int pe = e1 * 16 + e2;
            if (slot_of[pe] < 0) {
              slot_of[pe] = (int)pairs.size();
              pairs.push_back(pe);
              if (pool.size() < pairs.size()) pool.emplace_back();
              Acc &a = pool[(size_t)slot_of[pe]];
              if (a.val.size() < (size_t)D * D) {
                a.val.assign((size_t)D * D, 0.0);
                a.used.assign((size_t)D * D, 0);
              }
            }
            Acc &a = pool[(size_t)slot_of[pe]];
            const double c = p.coef * p.sl[e1] * p.sr[e2];
            auto add = [&](int si, int sj, double x) {
              const size_t idx = (size_t)(si + 1) * D + (sj + 1);
              if (!a.used[idx]) {
                a.used[idx] = 1;
                a.val[idx] = 0.0;
                a.touched.push_back((int)idx);
              }
              a.val[idx] += x;
            };
            if (var.type == 1) add(var.i, var.j, c);
            else for (const auto &t : var.lc) add(std::get<0>(t), std::get<1>(t), c * std::get<2>(t));
          }
        }
      }
      const Piece &p0 = in[(size_t)g[0]];
      const OpRef &var0 = side == 0 ? p0.l : p0.r;
      std::sort(pairs.begin(), pairs.end());
      for (int pe : pairs) {
        Acc &a = pool[(size_t)slot_of[pe]];
        slot_of[pe] = -1;
        std::sort(a.touched.begin(), a.touched.end());
        std::vector<std::tuple<int, int, double>> lc;
        for (int idx : a.touched) {
          a.used[(size_t)idx] = 0;
          const double x = a.val[(size_t)idx];
          if (x != 0.0) lc.emplace_back(idx / D - 1, idx % D - 1, x);
        }
        a.touched.clear();
        if (lc.empty()) continue;
        Piece q;
        q.coef = 1.0;
        q.hc = p0.hc;
        q.sl = mat_zero();
        q.sl[pe / 16] = 1.0;
        q.sr = mat_zero();
        q.sr[pe % 16] = 1.0;
        OpRef m = lincomb(var0.kind, var0.tr, lc);
        if (side == 0) { q.l = m; q.r = p0.r; } else { q.l = p0.l; q.r = m; }
        gout[gi].push_back(std::move(q));
      }
    }
  });
  std::vector<Piece> out;
  for (auto &v : gout) out.insert(out.end(), std::make_move_iterator(v.begin()), std::make_move_iterator(v.end()));
  return out;
}

std::vector<Piece> compress_pieces(std::vector<Piece> in) {
  return compress_side(compress_side(std::move(in), 0), 1);
}

// ---------------------------------------------------------------- new block ops

std::vector<NewOp> new_block_ops(const Integrals &I, int k, int side, const BlockLayout &nb,
                                 bool old_empty) {
  HalfOps O(&I, k, side == 0 ? old_empty : false, side == 1 ? old_empty : false);
  std::vector<NewOp> out;
  for (int f = 0; f < (int)nb.fam.size(); ++f) {
    const Family &F = nb.fam[f];
    for (int kk = 0; kk < F.K(); ++kk) {
      const int i = F.idx[kk][0], j = F.idx[kk][1];
      HalfOp d;
      if (side == 0) {
        switch (F.kind) {
          case KH: d = O.L_H(); break;
          case KC: d = O.L_C(i); break;
          case KT: d = O.L_T(i); break;
          case KA: d = O.L_A(i, j); break;
          case KB: d = O.L_B(i, j); break;
          default: throw std::runtime_error("bad kind for left block");
        }
      } else {
        switch (F.kind) {
          case KH: d = O.R_H(); break;
          case KC: d = O.R_C(i); break;
          case KV: d = O.R_V(i); break;
          case KA: d = O.R_A(i, j); break;
          case KB: d = O.R_B(i, j); break;
          default: throw std::runtime_error("bad kind for right block");
        }
      }
      if (old_empty) {
        HalfOp e;
        for (auto &x : d) if (x.blk.type == 0) e.push_back(x);
        d = e;
      }
      out.push_back({f, kk, d});
    }
  }
  return out;
}

// ---------------------------------------------------------------- dumps

static void dump_op(std::ostringstream &s, const OpRef &o) {
  if (o.type == 0) { s << "I"; return; }
  if (o.type == 1) { s << "S " << o.kind << ' ' << o.i << ' ' << o.j << ' ' << (int)o.tr; return; }
  s << "C " << o.kind << ' ' << (int)o.tr << ' ' << o.lc.size();
  char buf[64];
  for (auto &t : o.lc) {
    std::snprintf(buf, sizeof buf, " %d %d %.17g", std::get<0>(t), std::get<1>(t), std::get<2>(t));
    s << buf;
  }
}

static void dump_mat(std::ostringstream &s, const Mat4 &m) {
  char buf[32];
  for (double x : m) { std::snprintf(buf, sizeof buf, " %.17g", x); s << buf; }
}

std::string dump_pieces(const std::vector<Piece> &ps) {
  std::ostringstream s;
  char buf[64];
  for (auto &p : ps) {
    std::snprintf(buf, sizeof buf, "%.17g %d | ", p.coef, (int)p.hc);
    s << buf;
    dump_op(s, p.l);
    s << " |";
    dump_mat(s, p.sl);
    s << " |";
    dump_mat(s, p.sr);
    s << " | ";
    dump_op(s, p.r);
    s << '\n';
  }
  return s.str();
}

std::string dump_halfop(const HalfOp &h) {
  std::ostringstream s;
  char buf[64];
  for (auto &p : h) {
    std::snprintf(buf, sizeof buf, "%.17g | ", p.coef);
    s << buf;
    dump_op(s, p.blk);
    s << " |";
    dump_mat(s, p.site);
    s << '\n';
  }
  return s.str();
}

// ---------------------------------------------------------------- resolution

PreparedTemp prepare_temp(const BlockLayout &b, const OpRef &op) {
  PreparedTemp pt;
  std::vector<std::pair<int, double>> &m = pt.m;
  m.reserve(op.lc.size());
  for (auto &t : op.lc) {
    int f, kk;
    if (!b.get(op.kind, std::get<0>(t), std::get<1>(t), f, kk)) continue;
    if (pt.fam < 0) pt.fam = f;
    if (f != pt.fam) throw std::runtime_error("linear combination spans operator families");
    m.emplace_back(kk, std::get<2>(t));
  }
  if (m.empty()) return pt;
  pt.zero = false;
  // sources in (operator, coefficient) order, duplicates summed in that order
  if (!std::is_sorted(m.begin(), m.end())) std::sort(m.begin(), m.end());
  size_t w = 0;
  for (size_t r = 0; r < m.size(); ++r) {
    if (w > 0 && m[w - 1].first == m[r].first) m[w - 1].second += m[r].second;
    else m[w++] = m[r];
  }
  m.resize(w);
  uint64_t h = 0x243f6a8885a308d3ull;
  for (auto &x : m) {
    uint64_t bits;
    std::memcpy(&bits, &x.second, 8);
    h ^= (uint64_t)x.first + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h ^= bits + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  }
  pt.hash = h;
  return pt;
}

Ref TempSet::make(int side, const BlockLayout &b, const OpRef &op, bool &zero) {
  return make_prepared(side, b, op, prepare_temp(b, op), zero);
}

Ref TempSet::make_prepared(int side, const BlockLayout &b, const OpRef &op, PreparedTemp &&pt, bool &zero) {
  zero = pt.zero;
  if (pt.zero) return Ref();
  const int fam = pt.fam;
  auto fk = std::make_tuple(side, fam, op.tr);
  int tf;
  auto it = fam_of[side].find(fk);
  if (it == fam_of[side].end()) {
    TempFamily T;
    T.side = side;
    T.src_fam = fam;
    T.tr = op.tr;
    const Family &F = b.fam[fam];
    T.dnu = op.tr ? -F.dnu : F.dnu;
    T.dnd = op.tr ? -F.dnd : F.dnd;
    tf = (int)this->fam[side].size();
    this->fam[side].push_back(T);
    fam_of[side][fk] = tf;
  } else {
    tf = it->second;
  }
  // an identical temporary (same family, same sources, coefficients bit for bit)
  // is stored once
  auto same_bits = [](double x, double y) {
    uint64_t a, c;
    std::memcpy(&a, &x, 8);
    std::memcpy(&c, &y, 8);
    return a == c;
  };
  const std::vector<std::pair<int, double>> &m = pt.m;
  const uint64_t h = pt.hash ^ (((uint64_t)tf << 1) | (uint64_t)op.tr) * 0x9e3779b97f4a7c15ull;
  TempFamily &T = this->fam[side][tf];
  auto &cands = dedup[side][h];
  auto ref = [&](int kk) {
    Ref r;
    r.arena = 2 + side;
    r.fam = tf;
    r.k = kk;
    r.tr = false;
    r.dnu = T.dnu;
    r.dnd = T.dnd;
    r.par = (r.dnu + r.dnd) & 1;
    return r;
  };
  for (const auto &cand : cands) {
    if (cand.first != tf) continue;
    const auto &c = T.coefs[(size_t)cand.second];
    if (c.size() != m.size()) continue;
    bool eq = true;
    for (size_t i = 0; eq && i < m.size(); ++i) eq = c[i].first == m[i].first && same_bits(c[i].second, m[i].second);
    if (eq) return ref(cand.second);
  }
  const int kk = T.K();
  T.coefs.push_back(std::move(pt.m));
  cands.push_back({tf, kk});
  return ref(kk);
}

void TempSet::layout(const BlockLayout *blocks[2]) {
  for (int side = 0; side < 2; ++side) {
    int64_t cur = 0;
    for (auto &T : fam[side]) {
      const BlockLayout &b = *blocks[side];
      T.bra.assign(b.sec.size(), -1);
      T.off.assign(b.sec.size(), -1);
      T.base = cur;
      int64_t o = 0;
      for (int a = 0; a < (int)b.sec.size(); ++a) {
        const int br = b.find(b.sec[a].nu + T.dnu, b.sec[a].nd + T.dnd);
        T.bra[a] = br;
        if (br < 0) continue;
        T.off[a] = o;
        o += (int64_t)T.K() * b.sec[br].dim * b.sec[a].dim;
      }
      T.size = o;
      cur += o;
    }
    total[side] = cur;
  }
}

Ref resolve(const OpRef &op, int side, const BlockLayout &b, TempSet &temps, bool &zero) {
  zero = false;
  if (op.type == 0) return Ref();
  if (op.type == 1) {
    int f, kk;
    if (!b.get(op.kind, op.i, op.j, f, kk)) { zero = true; return Ref(); }
    Ref r;
    r.arena = side;
    r.fam = f;
    r.k = kk;
    r.tr = op.tr;
    const Family &F = b.fam[f];
    r.dnu = op.tr ? -F.dnu : F.dnu;
    r.dnd = op.tr ? -F.dnd : F.dnd;
    r.par = (r.dnu + r.dnd) & 1;
    return r;
  }
  return temps.make(side, b, op, zero);
}

bool prefer_transposed(int m, int n, int p, int q) {
  const double cn = (double)m * n * p + (double)m * p * q;
  const double ct = (double)n * p * q + (double)m * n * q;
  return ct < cn;
}

std::vector<int> stack_runs(const std::vector<uint64_t> &sorted_keys, int cap) {
  std::vector<int> runs;
  if (cap < 1) cap = 1;
  size_t k = 0;
  while (k < sorted_keys.size()) {
    int run = 1;
    while (run < cap && k + run < sorted_keys.size() && sorted_keys[k + run] == sorted_keys[k]) ++run;
    runs.push_back(run);
    k += run;
  }
  return runs;
}

KeptSet choose_kept(const std::vector<std::vector<double>> &ev_ascending, int mkeep, double drop) {
  struct Cand {
    double v;
    int e, j;
  };
  const int ne = (int)ev_ascending.size();
  KeptSet r;
  std::vector<Cand> cand;
  for (int e = 0; e < ne; ++e) {
    const int n = (int)ev_ascending[e].size();
    for (int j = 0; j < n; ++j) {
      const double x = ev_ascending[e][n - 1 - j];  // j-th largest in the sector
      cand.push_back({x, e, j});
      r.trace += x;
    }
  }
  std::stable_sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) {
    if (x.v != y.v) return x.v > y.v;
    if (x.e != y.e) return x.e < y.e;
    return x.j < y.j;
  });
  r.kept.assign(ne, 0);
  r.cols.assign(ne, {});
  // candidates above the drop threshold, and the first mkeep of them
  int nabove = 0;
  while (nabove < (int)cand.size() && cand[nabove].v > drop) ++nabove;
  const int n = std::max(0, std::min(mkeep, nabove));
  // a near-degenerate cluster across the cut: move the cut below the whole
  // cluster, unless nothing would be kept
  int nk = n;
  while (nk > 0 && nk < nabove && cand[nk - 1].v - cand[nk].v < kTruncCluster) --nk;
  if (nk == 0) nk = n;
  for (int i = 0; i < nk; ++i) {
    const Cand &c = cand[i];
    r.kept[c.e]++;
    r.kept_weight += c.v;
    r.cols[c.e].push_back((int)ev_ascending[c.e].size() - 1 - c.j);
  }
  r.cut_gap = std::numeric_limits<double>::infinity();
  if (nk > 0 && nk < nabove) r.cut_gap = cand[nk - 1].v - cand[nk].v;
  for (auto &c : r.cols) std::sort(c.begin(), c.end(), std::greater<int>());
  return r;
}

void pair_rdm(const std::vector<PsiBlockRef> &blocks, const double *psi, double rho[256]) {
  for (int i = 0; i < 256; ++i) rho[i] = 0.0;
  // blocks sharing the block sectors (a, d) couple; sum in block order
  std::map<std::pair<int, int>, std::vector<size_t>> by_ad;
  for (size_t i = 0; i < blocks.size(); ++i) by_ad[{blocks[i].a, blocks[i].d}].push_back(i);
  for (const auto &kv : by_ad)
    for (size_t u : kv.second)
      for (size_t w : kv.second) {
        const PsiBlockRef &s = blocks[u], &t = blocks[w];
        if (s.size != t.size) throw std::runtime_error("pair_rdm: blocks of one (a, d) differ in size");
        double acc = 0.0;
        for (int64_t e = 0; e < s.size; ++e) acc += psi[s.off + e] * psi[t.off + e];
        rho[(4 * s.b + s.c) * 16 + 4 * t.b + t.c] += acc;
      }
}

void small_symmetric_eigenvalues(int n, const double *a_in, double *ev) {
  if (n < 1 || n > 16) throw std::runtime_error("small_symmetric_eigenvalues: n out of range");
  double a[256];
  for (int i = 0; i < n * n; ++i) a[i] = a_in[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += a[i * n + j] * a[i * n + j];
    if (off <= 1e-30 * std::max(diag, 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (apq == 0.0) continue;
        // rotation angle that zeroes a_pq: tan(2 theta) = 2 a_pq / (a_qq - a_pp)
        const double tau = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - sn * akq;
          a[k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - sn * aqk;
          a[q * n + k] = sn * apk + c * aqk;
        }
      }
  }
  for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
  std::sort(ev, ev + n);
}

void orbital_entropies(const double rho[256], double out[3]) {
  double tr = 0.0;
  for (int i = 0; i < 16; ++i) tr += rho[i * 16 + i];
  if (!(tr > 0.0)) throw std::runtime_error("orbital_entropies: zero wave function");
  auto h = [](double x) { return x > 0.0 ? -x * std::log(x) : 0.0; };
  double sl = 0.0, sr = 0.0;
  for (int x = 0; x < 4; ++x) {
    double wl = 0.0, wr = 0.0;
    for (int y = 0; y < 4; ++y) {
      wl += rho[(4 * x + y) * 17];
      wr += rho[(4 * y + x) * 17];
    }
    sl += h(wl / tr);
    sr += h(wr / tr);
  }
  // the pair matrix is block diagonal in (n_up, n_dn) of the pair: diagonalise each block
  static const int NU[4] = {0, 1, 0, 1}, ND[4] = {0, 0, 1, 1};
  double spair = 0.0;
  for (int u = 0; u <= 2; ++u)
    for (int d = 0; d <= 2; ++d) {
      int idx[16], n = 0;
      for (int x = 0; x < 16; ++x)
        if (NU[x / 4] + NU[x % 4] == u && ND[x / 4] + ND[x % 4] == d) idx[n++] = x;
      if (n == 0) continue;
      double blk[256], ev[16];
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) blk[i * n + j] = rho[idx[i] * 16 + idx[j]] / tr;
      small_symmetric_eigenvalues(n, blk, ev);
      for (int i = 0; i < n; ++i) spair += h(ev[i]);
    }
  out[0] = sl;
  out[1] = sr;
  out[2] = spair;
}

}  // namespace dmrg
