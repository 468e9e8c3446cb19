// C ABI implementation: context, block storage, task lists and the FP64 path.
//
// Paper: Brabec et al., arXiv:2001.04890.  Sec. 2.1 (sweep, Eqs. renorm,
// h_mat, wf, wf_sec, renorm_mat, density matrices), Sec. 2.2.1 (H.psi task
// list, Eq. dgemm), Sec. 2.2.2 (renormalization task list and blocking
// tables), Sec. 2.2.3 (pre-summed operators, Eq. presum).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <functional>
#include <limits>
#include <map>
#include <cstring>
#include <exception>
#include <memory>
#include <utility>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dmrg_gb300.h"
#include "kernels.cuh"
#include "plan.hpp"

namespace dmrg {
void set_error(const std::string &s);

struct Fail {
  int code;
  std::string msg;
};

#define CK(x)                                                                              \
  do {                                                                                     \
    cudaError_t _e = (x);                                                                  \
    if (_e != cudaSuccess)                                                                 \
      throw Fail{_e == cudaErrorMemoryAllocation ? DMRG_ENOMEM : DMRG_ECUDA,               \
                 std::string(#x) + ": " + cudaGetErrorString(_e)};                         \
  } while (0)

#define CKS(x)                                                                             \
  do {                                                                                     \
    cusolverStatus_t _s = (x);                                                             \
    if (_s != CUSOLVER_STATUS_SUCCESS)                                                     \
      throw Fail{DMRG_ECUDA, std::string(#x) + ": cusolver status " + std::to_string(_s)}; \
  } while (0)

// ---------------------------------------------------------------- device buffers

// Allocator whose resize() leaves trivially constructible elements
// uninitialized: large host task lists are written once, by several threads,
// right after they are sized (no serial zero fill of fresh pages).
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U> &) noexcept {}
  template <class U, class... Args>
  void construct(U *p, Args &&...args) {
    ::new ((void *)p) U(std::forward<Args>(args)...);
  }
  template <class U>
  void construct(U *p) noexcept {
    ::new ((void *)p) U;
  }
};

// Host-side fault injection for the error paths: when positive, the n-th
// device allocation from now fails as if the device were out of memory
// (dmrg_debug_fail_alloc).  No GPU fault is involved.
static std::atomic<long long> g_fail_alloc_after{0};

static cudaError_t device_alloc(void **p, size_t bytes) {
  long long n = g_fail_alloc_after.load();
  while (n > 0) {
    if (g_fail_alloc_after.compare_exchange_weak(n, n - 1)) {
      if (n == 1) return cudaErrorMemoryAllocation;
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    CK(device_alloc(reinterpret_cast<void **>(&p), count * sizeof(T)));
    n = count;
  }
  template <class A>
  void upload(const std::vector<T, A> &h, cudaStream_t s) {
    alloc(h.size());
    if (!h.empty()) CK(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
};

static uint64_t eaddr(const double *p) { return (uint64_t)(uintptr_t)p / 8; }

// ---------------------------------------------------------------- enlarged layouts

struct ESub {
  int x, y, roff, m;  // left: (a, b); right: (c, d)
};
struct ESector {
  int nu, nd, dim;
  std::vector<ESub> sub;
};
using Enlarged = std::vector<ESector>;

static Enlarged enlarged(const BlockLayout &b, int direction) {
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> groups;
  for (int a = 0; a < (int)b.sec.size(); ++a)
    for (int s = 0; s < 4; ++s) {
      const std::pair<int, int> E{b.sec[a].nu + SITE_NU[s], b.sec[a].nd + SITE_ND[s]};
      if (direction > 0) groups[E].push_back({a, s});
      else groups[E].push_back({s, a});
    }
  Enlarged out;
  for (auto &g : groups) {
    ESector es;
    es.nu = g.first.first;
    es.nd = g.first.second;
    std::sort(g.second.begin(), g.second.end());
    int off = 0;
    for (auto &xy : g.second) {
      const int m = direction > 0 ? b.sec[xy.first].dim : b.sec[xy.second].dim;
      es.sub.push_back({xy.first, xy.second, off, m});
      off += m;
    }
    es.dim = off;
    out.push_back(es);
  }
  return out;
}

// ---------------------------------------------------------------- blocks

struct DevBlock {
  BlockLayout lay;
  DBuf<double> ops;  // all stored families
  // the renormalization that produced this block (for the wave-function prediction)
  Enlarged parent;
  std::vector<int> kept;
  std::vector<int64_t> Ooff;
  DBuf<double> O;
  const double *arena() const { return ops.p; }
};

struct PsiBlock {
  int a, b, c, d, ma, md;
  int64_t off;
};

struct Psi {
  std::vector<PsiBlock> blk;
  std::vector<int> index;  // ((a*4+b)*4+c)*nr+d -> block or -1
  int nl = 0, nr = 0;
  int64_t dim = 0;
  int find(int a, int b, int c, int d) const {
    if (a < 0 || d < 0 || a >= nl || d >= nr) return -1;
    return index[((a * 4 + b) * 4 + c) * nr + d];
  }
  int find_block(uint64_t off) const {  // block index by element offset (-1 if none)
    const auto it = std::lower_bound(blk.begin(), blk.end(), (int64_t)off,
                                     [](const PsiBlock &b, int64_t o) { return b.off < o; });
    return it != blk.end() && it->off == (int64_t)off ? (int)(it - blk.begin()) : -1;
  }
};

static Psi psi_layout(const BlockLayout &l, const BlockLayout &r, int nu, int nd) {
  Psi P;
  P.nl = (int)l.sec.size();
  P.nr = (int)r.sec.size();
  P.index.assign((size_t)P.nl * 16 * P.nr, -1);
  int64_t off = 0;
  for (int a = 0; a < P.nl; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c)
        for (int d = 0; d < P.nr; ++d) {
          const int u = l.sec[a].nu + SITE_NU[b] + SITE_NU[c] + r.sec[d].nu;
          const int v = l.sec[a].nd + SITE_ND[b] + SITE_ND[c] + r.sec[d].nd;
          if (u != nu || v != nd) continue;
          P.index[((a * 4 + b) * 4 + c) * P.nr + d] = (int)P.blk.size();
          P.blk.push_back({a, b, c, d, l.sec[a].dim, r.sec[d].dim, off});
          off += (int64_t)l.sec[a].dim * r.sec[d].dim;
        }
  P.dim = off;
  return P;
}

// resolved operator -> effective block for ket sector a
struct Arenas {
  const BlockLayout *lay[2];
  const void *stored[2];
  const TempSet *temps;
  const void *temp[2];
  int esize;  // bytes per element of the arenas (8: FP64 masters, 4: FP32 copies)
};

static bool eff_block(const Ref &r, const Arenas &A, int side, int a, int &a2, uint64_t &addr,
                      int &rs, int &cs) {
  const BlockLayout &b = *A.lay[side];
  if (r.arena < 0) {
    a2 = a;
    addr = ~0ull;
    rs = cs = 0;
    return true;
  }
  const std::vector<int> *bra;
  const std::vector<int64_t> *off;
  int64_t base;
  int dnu, dnd;
  const void *arena;
  bool tr = r.tr;
  if (r.arena < 2) {
    const Family &F = b.fam[r.fam];
    bra = &F.bra;
    off = &F.off;
    base = F.base;
    dnu = F.dnu;
    dnd = F.dnd;
    arena = A.stored[side];
  } else {
    const TempFamily &T = A.temps->fam[side][r.fam];
    bra = &T.bra;
    off = &T.off;
    base = T.base;
    dnu = T.dnu;
    dnd = T.dnd;
    arena = A.temp[side];
  }
  const int ma = b.sec[a].dim;
  if (!tr) {
    a2 = (*bra)[a];
    if (a2 < 0) return false;
    const int m2 = b.sec[a2].dim;
    addr = (uint64_t)(uintptr_t)arena / A.esize + base + (*off)[a] + (int64_t)r.k * m2 * ma;
    rs = ma;
    cs = 1;
  } else {
    const int ket = b.find(b.sec[a].nu - dnu, b.sec[a].nd - dnd);
    if (ket < 0 || (*bra)[ket] != a) return false;
    a2 = ket;
    const int m2 = b.sec[ket].dim;
    addr = (uint64_t)(uintptr_t)arena / A.esize + base + (*off)[ket] + (int64_t)r.k * ma * m2;
    rs = 1;
    cs = m2;
  }
  return true;
}

static int site_image(const Mat4 &S, int b, double &val) {
  for (int r = 0; r < 4; ++r)
    if (S[r * 4 + b] != 0.0) {
      val = S[r * 4 + b];
      return r;
    }
  return -1;
}

static inline int npart(const Sector &s) { return s.nu + s.nd; }
static inline int nsite(int b) { return SITE_NU[b] + SITE_ND[b]; }

// task list grouped by output block
struct ChainList {
  using Keyed = std::vector<std::pair<int, ChainEntry>>;  // (group key, entry)
  Keyed ent;                    // entries in build order
  std::vector<Keyed> parts;     // further entries, built after ent, in part order
  std::vector<ChainGroup> grp;  // one per key, filled by finish()
  std::vector<ChainEntry, NoInitAlloc<ChainEntry>> flat;
  int ntiles = 0;
  double flops = 0.0;
  size_t size() const {
    size_t n = ent.size();
    for (const auto &p : parts) n += p.size();
    return n;
  }
  // Group the tasks by output block: a stable counting sort on the group key
  // (keys index protos), groups in key order, tasks in build order within one
  // (ent, then the parts in order).  Each part is counted and scattered by its
  // own thread: per (part, key) write offsets keep the order of a serial sort.
  void finish(const std::vector<ChainGroup> &protos) {
    const size_t ng = protos.size();
    std::vector<const Keyed *> src{&ent};
    for (const auto &p : parts) src.push_back(&p);
    const size_t ns = src.size();
    std::vector<int64_t> cnt(ns * ng, 0);
    parallel_for(ns, [&](size_t s) {
      int64_t *c = cnt.data() + s * ng;
      for (const auto &pe : *src[s]) ++c[(size_t)pe.first];
    });
    std::vector<int64_t> start(ng + 1, 0), off(ns * ng);
    int64_t run = 0;
    for (size_t k = 0; k < ng; ++k) {
      start[k] = run;
      for (size_t s = 0; s < ns; ++s) {
        off[s * ng + k] = run;
        run += cnt[s * ng + k];
      }
    }
    start[ng] = run;
    flat.clear();
    flat.resize((size_t)run);  // every element is written by the scatter below
    parallel_for(ns, [&](size_t s) {
      int64_t *o = off.data() + s * ng;
      for (const auto &pe : *src[s]) flat[(size_t)o[(size_t)pe.first]++] = pe.second;
    });
    Keyed().swap(ent);  // the grouped copy is all that is used
    std::vector<Keyed>().swap(parts);
    grp.clear();
    ntiles = 0;
    for (size_t k = 0; k < ng; ++k) {
      const int64_t c = start[k + 1] - start[k];
      if (c == 0) continue;
      ChainGroup g = protos[k];
      g.first = (int)start[k];
      g.count = (int)c;
      g.tile0 = ntiles;
      ntiles += ((g.m + 31) / 32) * ((g.q + 31) / 32);
      grp.push_back(g);
    }
  }
};

static double entry_flops(int m, int n, int p, int q, bool xid, bool zid);

// Launch-shape parameters of a task list, chosen by dmrg_autotune: the split
// granularity (about target_chunks chunks, none lighter than min_chunk FLOPs)
// the smallest output-block side routed to the tensor cores, and the launch
// order of the groups.
struct ChainTune {
  double target_chunks = 8192.0;
  double min_chunk = 2.0e5;
  int tc_min = 33;
  int by_work = 0;     // 1: launch groups heaviest first; 0: in output-block order (operand locality)
  int orient = 1;      // run each entry in its cheaper association (split task lists)
  int flat_wide = 1;   // flat kernel CTAs: 1 = one wide CTA per SM (6 FP64 / 12 FP32 warps),
                       // 0 = two narrower CTAs per SM (4 / 8 warps each)
  int tc_tiny = 0;     // tensor-core kernel shapes: 1 = every block that fits the 32-column
                       // shape runs on it (a launch of its own), 0 = only when all blocks fit
};
// Host half of a task list's upload: the execution list (entries in their
// cheaper association, cut into equal-work chunks when split_tasks), the launch
// groups of the three chunk kernels (32 x 32 tiles, flattened lanes, tensor
// cores) and the ordered reduction of the chunk slots.
struct ExecPlan {
  std::vector<ChainEntry, NoInitAlloc<ChainEntry>> xs;
  std::vector<double, NoInitAlloc<double>> w;
  std::vector<ChainGroup> vb, vf, vt;
  std::vector<ReduceGroup> vr;
  int tiles = 0;
  int64_t soff = 0, e0 = 0;
};

// The entry D^T += f Z^T Y^T X^T of D += f X Y Z: same operands, swapped strides.
static ChainEntry transposed_entry(const ChainEntry &e) {
  ChainEntry t{};
  t.x = e.z;  // X' = Z^T
  t.xrs = e.zcs;
  t.xcs = e.zrs;
  t.y = e.y;  // Y' = Y^T
  t.yrs = e.ycs;
  t.ycs = e.yrs;
  t.z = e.x;  // Z' = X^T
  t.zrs = e.xcs;
  t.zcs = e.xrs;
  t.n = e.p;
  t.p = e.n;
  t.f = e.f;
  return t;
}

static void plan_exec(const ChainList &CL, bool tensor_cores, bool split_tasks, const ChainTune &tune,
                      ExecPlan &X) {
  std::vector<ChainGroup> &vb = X.vb, &vf = X.vf, &vt = X.vt;
  std::vector<ReduceGroup> &vr = X.vr;
  int &tiles = X.tiles;
  int64_t &soff = X.soff, &e0 = X.e0;
  tiles = 0;
  soff = e0 = 0;
  auto &xs = X.xs;
  auto &w = X.w;
  auto tc_entry_ok = [&](const ChainEntry &e, int m, int q) {
    // Y must be a whole row-major psi block; identity sides are square
    return !(e.n < 1 || e.p < 1 || e.n > 128 || e.p > 128 || e.y == ~0ull || e.ycs != 1 || e.yrs != e.p ||
             (e.x == ~0ull && e.n != m) || (e.z == ~0ull && e.p != q));
  };
  auto tc_shape_ok = [&](int m, int q) {
    return tensor_cores && m <= 128 && q <= 128 && (m >= tune.tc_min || q >= tune.tc_min);
  };
  auto weight = [](const ChainGroup &g, const ChainEntry &e) {
    return 1.0 + entry_flops(g.m, e.n, e.p, g.q, e.x == ~0ull, e.z == ~0ull);
  };
  // chunk kind: tensor-core chunks need every entry in the tensor-core form
  auto place = [&](ChainGroup t, bool entries_tc_ok) {
    if (t.count > 0 && tc_shape_ok(t.m, t.q) && entries_tc_ok) {
      vt.push_back(t);
    } else if (t.m <= 32 && t.q <= 32) {
      vf.push_back(t);
    } else {
      t.tile0 = tiles;
      tiles += ((t.m + 31) / 32) * ((t.q + 31) / 32);
      vb.push_back(t);
    }
  };
  auto chunk_tc_ok = [&](const ChainGroup &t) {
    bool ok = t.count > 0 && tc_shape_ok(t.m, t.q);
    for (int i = t.first; ok && i < t.first + t.count; ++i) ok = tc_entry_ok(xs[i], t.m, t.q);
    return ok;
  };
  const size_t ng = CL.grp.size();
  if (!split_tasks) {
    xs.reserve(CL.flat.size());
    w.reserve(CL.flat.size());
    for (const auto &g : CL.grp) {
      ChainGroup t = g;
      t.first = (int)xs.size();
      for (int i = g.first; i < g.first + g.count; ++i) {
        xs.push_back(CL.flat[i]);
        w.push_back(weight(g, CL.flat[i]));
      }
      place(t, chunk_tc_ok(t));
    }
  } else {
    // Execution list: the entries of an output block whose other association
    // is cheaper (n p q + m n q < m n p + m p q) run as the transposed product
    // in chunks of their own, after the block's other chunks; their slot is
    // written through transposed strides, so the ordered reduction is
    // unchanged.  Tensor-core blocks keep the stored association.  Output
    // blocks are planned in parallel; every weight is an integer, so the sums
    // (and with them the chunk boundaries) do not depend on the order.
    std::vector<double> gwork(ng, 0.0);
    parallel_for(ng, [&](size_t gi) {
      const ChainGroup &g = CL.grp[gi];
      double a = 0.0;
      for (int i = g.first; i < g.first + g.count; ++i) a += weight(g, CL.flat[i]);
      gwork[gi] = a;
    });
    double total = 0.0;
    for (double a : gwork) total += a;
    const double chunk_work = std::max(total / tune.target_chunks, tune.min_chunk);
    struct GroupExec {
      bool tc = false;                 // tensor-core shape with every entry in tensor-core form
      int nn = 0;                      // entries kept in the stored association
      std::vector<int> csize[2];       // chunk sizes: stored association, transposed
      std::vector<char> ctc[2];        // chunk routable to the tensor cores (filled with the entries)
      int64_t xbase = 0, soff = 0;
    };
    std::vector<GroupExec> ge(ng);
    auto transposed_here = [&](const ChainGroup &g, bool tcg, const ChainEntry &e) {
      return tune.orient && !tcg && e.x != ~0ull && e.z != ~0ull && prefer_transposed(g.m, e.n, e.p, g.q);
    };
    parallel_for(ng, [&](size_t gi) {
      const ChainGroup &g = CL.grp[gi];
      GroupExec &G = ge[gi];
      bool tcg = tc_shape_ok(g.m, g.q);
      for (int i = g.first; tcg && i < g.first + g.count; ++i) tcg = tc_entry_ok(CL.flat[i], g.m, g.q);
      G.tc = tcg;
      for (int part = 0; part < 2; ++part) {
        // greedy equal-work chunks over this part's entries, in build order
        double acc = 0.0;
        int cnt = 0;
        for (int i = g.first; i < g.first + g.count; ++i) {
          const ChainEntry &e = CL.flat[i];
          if (transposed_here(g, tcg, e) != (part == 1)) continue;
          if (part == 0) ++G.nn;
          const double we = part == 0 ? weight(g, e) : 1.0 + entry_flops(g.q, e.p, e.n, g.m, false, false);
          if (cnt > 0 && acc + we > chunk_work) {
            G.csize[part].push_back(cnt);
            acc = 0.0;
            cnt = 0;
          }
          acc += we;
          ++cnt;
        }
        if (cnt > 0) G.csize[part].push_back(cnt);
      }
    });
    int64_t nx = 0;
    for (size_t gi = 0; gi < ng; ++gi) {
      const ChainGroup &g = CL.grp[gi];
      ge[gi].xbase = nx;
      ge[gi].soff = soff;
      nx += g.count;
      soff += (int64_t)(ge[gi].csize[0].size() + ge[gi].csize[1].size()) * g.m * g.q;
    }
    xs.resize((size_t)nx);  // every element is written below
    w.resize((size_t)nx);
    parallel_for(ng, [&](size_t gi) {
      const ChainGroup &g = CL.grp[gi];
      GroupExec &G = ge[gi];
      int64_t a = G.xbase, b = G.xbase + G.nn;
      for (int i = g.first; i < g.first + g.count; ++i) {
        const ChainEntry &e = CL.flat[i];
        if (!transposed_here(g, G.tc, e)) {
          xs[(size_t)a] = e;
          w[(size_t)a++] = weight(g, e);
        } else {
          const ChainEntry t = transposed_entry(e);
          xs[(size_t)b] = t;
          w[(size_t)b++] = 1.0 + entry_flops(g.q, t.n, t.p, g.m, false, false);
        }
      }
      int64_t first = G.xbase;
      for (int part = 0; part < 2; ++part)
        for (int c : G.csize[part]) {
          ChainGroup t{};
          t.first = (int)first;
          t.count = c;
          t.m = part == 0 ? g.m : g.q;
          t.q = part == 0 ? g.q : g.m;
          G.ctc[part].push_back(chunk_tc_ok(t) ? 1 : 0);
          first += c;
        }
    });
    for (size_t gi = 0; gi < ng; ++gi) {
      const ChainGroup &g = CL.grp[gi];
      const GroupExec &G = ge[gi];
      const int64_t mq = (int64_t)g.m * g.q;
      ReduceGroup r{};
      r.e0 = e0;
      r.soff = G.soff;
      r.d = g.d;
      r.drs = g.drs;
      r.dcs = g.dcs;
      r.m = g.m;
      r.q = g.q;
      int nsplit = 0;
      int64_t first = G.xbase;
      for (int part = 0; part < 2; ++part)
        for (size_t c = 0; c < G.csize[part].size(); ++c) {
          ChainGroup t = g;
          t.first = (int)first;
          t.count = G.csize[part][c];
          t.d = (uint64_t)(G.soff + (int64_t)nsplit * mq);  // slot: m x q row-major
          if (part == 0) {
            t.drs = g.q;
            t.dcs = 1;
          } else {  // transposed chunk: q x m output written into the m x q slot
            t.m = g.q;
            t.q = g.m;
            t.drs = 1;
            t.dcs = g.q;
          }
          place(t, G.ctc[part][c] != 0);
          ++nsplit;
          first += t.count;
        }
      r.nsplit = nsplit;
      vr.push_back(r);
      e0 += mq;
    }
  }
  // optionally heaviest groups first: CTAs are dispatched in grid order, so the
  // light groups fill the last wave; the natural order keeps the chunks of one
  // output block (which read the same operators) adjacent.  Results do not
  // depend on the order.
  auto by_work = [&](std::vector<ChainGroup> &v) {
    std::vector<std::pair<double, int>> key(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      double wsum = 0.0;
      for (int e = v[i].first; e < v[i].first + v[i].count; ++e) wsum += w[e];
      key[i] = {-wsum, (int)i};
    }
    std::stable_sort(key.begin(), key.end());
    std::vector<ChainGroup> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[key[i].second];
    v.swap(out);
  };
  if (tune.by_work) {
    by_work(vf);
    by_work(vt);
  }
}

// First-use numbering of keys: occurrence i (0 <= i < n < 2^32) has key
// key_of(i); uid[i] receives the number of its key, keys numbered in order of
// first occurrence, and first[u] the first occurrence of key u.  Parallel: the
// keys are split into hash shards; the occurrences of each shard are listed in
// increasing order (a counting pass per chunk of occurrences, then a scatter),
// each shard is numbered by one thread, and the shards' first occurrences are
// merged into one increasing list, so the numbering is that of a serial pass.
template <class Key, class Hash, class KeyOf>
static void first_use_numbering(size_t n, KeyOf key_of, Hash hash, std::vector<uint32_t> &uid,
                                std::vector<size_t> &first) {
  const size_t S = 16, B = 1 << 16;
  if (n >= (size_t(1) << 32)) throw Fail{DMRG_EINVAL, "too many occurrences to number"};
  const size_t nc = (n + B - 1) / B;
  std::vector<uint8_t> shard(n);
  std::vector<uint32_t> ccount(nc * S, 0);  // occurrences of each shard in each chunk
  parallel_for(nc, [&](size_t c) {
    uint32_t *cnt = &ccount[c * S];
    for (size_t i = c * B; i < std::min(n, (c + 1) * B); ++i) {
      const uint8_t sh = (uint8_t)((hash(key_of(i)) >> 40) % S);
      shard[i] = sh;
      ++cnt[sh];
    }
  });
  // occ[sstart[sh] ..] lists shard sh's occurrences in increasing order (chunk by chunk)
  std::vector<size_t> sstart(S + 1, 0), coff(nc * S);
  for (size_t sh = 0; sh < S; ++sh) {
    size_t acc = 0;
    for (size_t c = 0; c < nc; ++c) {
      coff[c * S + sh] = acc;
      acc += ccount[c * S + sh];
    }
    sstart[sh + 1] = sstart[sh] + acc;
  }
  std::vector<uint32_t> occ(n);
  parallel_for(nc, [&](size_t c) {
    size_t w[S];
    for (size_t sh = 0; sh < S; ++sh) w[sh] = sstart[sh] + coff[c * S + sh];
    for (size_t i = c * B; i < std::min(n, (c + 1) * B); ++i) occ[w[shard[i]]++] = (uint32_t)i;
  });
  std::vector<uint32_t> lid(n);
  std::vector<std::vector<size_t>> lfirst(S);
  parallel_for(S, [&](size_t sh) {
    // open-addressing table (linear probing, at most half full)
    struct Slot {
      Key key;
      uint64_t h;
      uint32_t id;
    };
    const uint32_t EMPTY = 0xffffffffu;
    std::vector<Slot> tab(1024, Slot{Key{}, 0, EMPTY});
    size_t used = 0;
    auto place = [&](std::vector<Slot> &t, const Slot &x) {
      size_t at = (size_t)x.h & (t.size() - 1);
      while (t[at].id != EMPTY) at = (at + 1) & (t.size() - 1);
      t[at] = x;
    };
    for (size_t qi = sstart[sh]; qi < sstart[sh + 1]; ++qi) {
      const size_t i = occ[qi];
      const Key k = key_of(i);
      const uint64_t h = (uint64_t)hash(k);
      size_t at = (size_t)h & (tab.size() - 1);
      while (tab[at].id != EMPTY && !(tab[at].h == h && tab[at].key == k)) at = (at + 1) & (tab.size() - 1);
      if (tab[at].id != EMPTY) {
        lid[i] = tab[at].id;
        continue;
      }
      const uint32_t id = (uint32_t)lfirst[sh].size();
      lfirst[sh].push_back(i);
      lid[i] = id;
      tab[at] = Slot{k, h, id};
      if (2 * ++used > tab.size()) {
        std::vector<Slot> bigger(2 * tab.size(), Slot{Key{}, 0, EMPTY});
        for (const Slot &x : tab)
          if (x.id != EMPTY) place(bigger, x);
        tab.swap(bigger);
      }
    }
  });
  // global numbers in order of first occurrence: merge the shards' increasing lists
  std::vector<std::vector<uint32_t>> gnum(S);
  std::vector<size_t> pos(S, 0);
  size_t keys = 0;
  for (size_t sh = 0; sh < S; ++sh) {
    gnum[sh].resize(lfirst[sh].size());
    keys += lfirst[sh].size();
  }
  first.clear();
  first.reserve(keys);
  for (size_t u = 0; u < keys; ++u) {
    size_t bsh = S, best = n;
    for (size_t sh = 0; sh < S; ++sh)
      if (pos[sh] < lfirst[sh].size() && lfirst[sh][pos[sh]] < best) {
        best = lfirst[sh][pos[sh]];
        bsh = sh;
      }
    gnum[bsh][pos[bsh]++] = (uint32_t)first.size();
    first.push_back(best);
  }
  uid.resize(n);
  parallel_for((n + B - 1) / B, [&](size_t c) {
    for (size_t i = c * B; i < std::min(n, (c + 1) * B); ++i) uid[i] = gnum[shard[i]][lid[i]];
  });
}

// An operator view read as a tensor-core tile: source address, strides, shape.
struct ViewKey {
  uint64_t src;
  int rs, cs, R, K;
  bool operator==(const ViewKey &o) const {
    return src == o.src && rs == o.rs && cs == o.cs && R == o.R && K == o.K;
  }
};
struct ViewHash {
  size_t operator()(const ViewKey &k) const {
    uint64_t h = k.src * 0x9E3779B97F4A7C15ull;
    h ^= ((uint64_t)(uint32_t)k.rs << 32 | (uint32_t)k.cs) + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
    h ^= ((uint64_t)(uint32_t)k.R << 32 | (uint32_t)k.K) + 0x8CB92BA72F3D8DD7ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};
struct OffsetHash {
  size_t operator()(uint64_t y) const {
    uint64_t h = y * 0x9E3779B97F4A7C15ull;
    return (size_t)(h ^ (h >> 29));
  }
};

// Host plan of the tensor-core launch: entries with tile offsets, blocks
// ordered by kernel shape, and the operator-view and psi tiles to build.
// Tiles are laid out in order of first use in launch order; identical views
// are stored once (deduplicated by address, strides and shape); identity
// operators are exact identity tiles.
struct TcPlan {
  std::vector<TcEntry> te;
  std::vector<TcGroup> tg;
  std::vector<TileSpec> ts;
  std::vector<PsiTileSpec> ps;
  int ntc_shape[3] = {0, 0, 0};
  uint64_t opbytes = 0, psibytes = 0;
};

static void plan_tc(const std::vector<ChainEntry, NoInitAlloc<ChainEntry>> &xs, const std::vector<ChainGroup> &vt,
                    TcPlan &P, std::vector<int> *entry_of = nullptr, uint64_t elem_bytes = 4, int tc_tiny = 0) {
  auto c16 = [](int x) { return (uint64_t)((x + 15) & ~15); };
  const size_t nv = vt.size();
  // kernel shape per block: 2 (m <= 64, q, p <= 32), 1 (m, q, p <= 64), 0 (the rest);
  // blocks ordered by shape.  Shape 2 is used when every block fits it, or for every
  // block that fits it with tc_tiny: each shape is its own launch with its own
  // last-wave tail, and whether a third launch costs more than its extra resident
  // CTAs gain depends on the mix of block sizes (an autotuner candidate).
  std::vector<int> pmax(nv, 0);
  parallel_for(nv, [&](size_t i) {
    const ChainGroup &g = vt[i];
    int m = 0;
    for (int j = g.first; j < g.first + g.count; ++j) m = std::max(m, xs[j].p);
    pmax[i] = m;
  });
  auto fits = [&](size_t i, int lim_q) { return vt[i].m <= 64 && vt[i].q <= lim_q && pmax[i] <= lim_q; };
  bool all_tiny = true;
  for (size_t i = 0; i < nv; ++i) all_tiny = all_tiny && fits(i, 32);
  auto shape_of = [&](size_t i) {
    if (all_tiny || (tc_tiny && fits(i, 32))) return 2;
    return fits(i, 64) ? 1 : 0;
  };
  std::vector<size_t> order;
  for (int sh : {2, 1, 0}) {
    int cnt = 0;
    for (size_t i = 0; i < nv; ++i)
      if (shape_of(i) == sh) {
        order.push_back(i);
        ++cnt;
      }
    P.ntc_shape[sh] = cnt;
  }
  const size_t nb = order.size();
  std::vector<int64_t> base(nb + 1, 0);
  for (size_t k = 0; k < nb; ++k) base[k + 1] = base[k] + vt[order[k]].count;
  const size_t T = (size_t)base[nb];
  P.tg.resize(nb);
  P.te.assign(T, TcEntry{});
  std::vector<int> src(T), blk(T);  // per launch position: entry index, block
  parallel_for(nb, [&](size_t k) {
    const ChainGroup &g = vt[order[k]];
    P.tg[k] = TcGroup{g.d, g.drs, g.dcs, g.m, g.q, (int)base[k], g.count};
    // tasks of this output block that read the same psi block run as stacks: their X
    // along the MMA's M in one stage 1 (at most MR / m16 of them, MR the shape's M)
    const int mr = shape_of(order[k]) == 0 ? 128 : 64;
    const int cap = std::max(1, std::min(8, mr / (int)c16(g.m)));
    std::vector<int> idx(g.count);
    std::iota(idx.begin(), idx.end(), g.first);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return xs[a].y < xs[b].y; });
    std::vector<uint64_t> keys(idx.size());
    for (size_t j = 0; j < idx.size(); ++j) keys[j] = xs[idx[j]].y;
    const std::vector<int> runs = stack_runs(keys, cap);
    size_t run_i = 0;
    int remaining = 0;
    for (size_t j = 0; j < idx.size(); ++j) {
      const ChainEntry &e = xs[idx[j]];
      TcEntry &t = P.te[(size_t)base[k] + j];
      if (remaining == 0) {  // first member of a stack: the run of tasks on this psi block
        t.stack = (uint8_t)runs[run_i++];
        remaining = t.stack;
      }
      --remaining;
      t.n = (uint8_t)e.n;
      t.p = (uint8_t)e.p;
      t.f = (float)e.f;
      src[(size_t)base[k] + j] = idx[j];
      blk[(size_t)base[k] + j] = (int)k;
    }
  });
  // operator views: occurrence 2 i is entry i's X, 2 i + 1 its Z^T
  auto view_of = [&](size_t o) {
    const size_t i = o >> 1;
    const ChainEntry &e = xs[(size_t)src[i]];
    const TcGroup &g = P.tg[(size_t)blk[i]];
    if ((o & 1) == 0)
      return e.x == ~0ull ? ViewKey{~0ull, 0, 0, e.n, e.n} : ViewKey{e.x * elem_bytes, e.xrs, e.xcs, g.m, e.n};
    return e.z == ~0ull ? ViewKey{~0ull, 0, 0, e.p, e.p} : ViewKey{e.z * elem_bytes, e.zcs, e.zrs, g.q, e.p};
  };
  std::vector<uint32_t> vid;
  std::vector<size_t> vfirst;
  first_use_numbering<ViewKey>(2 * T, view_of, ViewHash(), vid, vfirst);
  std::vector<uint64_t> voff(vfirst.size());
  for (size_t u = 0; u < vfirst.size(); ++u) {
    const ViewKey v = view_of(vfirst[u]);
    voff[u] = P.opbytes;
    P.ts.push_back(TileSpec{v.src, P.opbytes, v.rs, v.cs, v.R, v.K});
    P.opbytes += c16(v.R) * c16(v.K) * 4;
  }
  // psi blocks read as Y^T
  auto y_of = [&](size_t i) { return xs[(size_t)src[i]].y; };
  std::vector<uint32_t> yid;
  std::vector<size_t> yfirst;
  first_use_numbering<uint64_t>(T, y_of, OffsetHash(), yid, yfirst);
  std::vector<uint64_t> yoff(yfirst.size());
  for (size_t u = 0; u < yfirst.size(); ++u) {
    const ChainEntry &e = xs[(size_t)src[yfirst[u]]];
    yoff[u] = P.psibytes;
    P.ps.push_back(PsiTileSpec{(int64_t)e.y, P.psibytes, e.n, e.p});
    P.psibytes += c16(e.p) * c16(e.n) * 4;
  }
  if (P.psibytes >= (1ull << 32)) throw Fail{DMRG_EINVAL, "psi tiles exceed the 4 GiB a task descriptor addresses"};
  parallel_for((T + 65535) / 65536, [&](size_t c) {
    for (size_t i = c * 65536; i < std::min(T, (c + 1) * 65536); ++i) {
      P.te[i].xt = voff[vid[2 * i]];
      P.te[i].zt = voff[vid[2 * i + 1]];
      P.te[i].yt = (uint32_t)yoff[yid[i]];
    }
  });
  if (entry_of) entry_of->swap(src);
}

// A task list on the device.  When the tensor cores are enabled, output blocks
// with both sides <= 128, one side >= tc_min and every entry's n, p <= 128 go
// to the tensor-core kernel; of the rest, blocks of at most 32 x 32 go to the
// flattened-lane warp kernel and larger ones to the 32 x 32 tile kernel.  With
// split_tasks, every output block's entry list is cut into
// chunks of about equal work; each chunk accumulates into its own slot of a
// scratch buffer and a reduction adds the slots in chunk order, so the result
// does not depend on scheduling (bitwise repeatable) while the grid has
// thousands of independent tasks.
struct DevChain {
  DBuf<ChainEntry> ent, xent;
  DBuf<ChainGroup> all, big, flat;
  DBuf<ReduceGroup> red;
  DBuf<double> scratch;
  // tensor-core groups: entries with pre-split operand tiles (operators tiled
  // once here, the psi blocks they read re-tiled at every launch)
  DBuf<TcEntry> tce;
  DBuf<TcGroup> tcg;  // blocks ordered by kernel shape: 2, 1, 0 (ntc_shape[] of each)
  DBuf<PsiTileSpec> pts;
  DBuf<uint8_t> optiles, psitiles;
  DBuf<int> tc_counter;  // work counters of the persistent tensor-core kernels (two shapes)
  int npts = 0, ntc_shape[3] = {0, 0, 0};
  int flat_wide = 1;
  int tc_tiny = 0;
  int nall = 0, nbig = 0, nflat = 0, ntc = 0, ntiles = 0, nred = 0;
  int64_t nent = 0;
  int64_t red_total = 0, scratch_n = 0;
  bool split = false;
  bool ops32 = false;  // X and Z operands are FP32 copies (else the FP64 masters)

  void upload(const ChainList &CL, cudaStream_t s, bool tensor_cores = false, bool split_tasks = false,
              const ChainTune &tune = ChainTune(), bool ops32_in = false) {
    ExecPlan X;
    plan_exec(CL, tensor_cores, split_tasks, tune, X);
    split = split_tasks;
    ops32 = ops32_in;
    flat_wide = tune.flat_wide;
    tc_tiny = tune.tc_tiny;
    const auto &xs = X.xs;
    const std::vector<ChainGroup> &vb = X.vb, &vf = X.vf, &vt = X.vt;
    const std::vector<ReduceGroup> &vr = X.vr;
    const int tiles = X.tiles;
    const int64_t soff = X.soff, e0 = X.e0;
    ent.upload(CL.flat, s);  // the task list as built (diagonal, batching)
    xent.upload(xs, s);      // the execution list of the chunk kernels
    nent = (int64_t)CL.flat.size();
    all.upload(CL.grp, s);
    big.upload(vb, s);
    flat.upload(vf, s);
    build_tc(xs, vt, s);
    red.upload(vr, s);
    nall = (int)CL.grp.size();
    nbig = (int)vb.size();
    nflat = (int)vf.size();
    nred = (int)vr.size();
    ntiles = tiles;
    red_total = e0;
    scratch_n = soff;
    if (split) scratch.alloc((size_t)std::max<int64_t>(soff, 1));
  }

  // Tensor-core entries: tile images of every X, Z^T operator view (deduplicated,
  // exact identity tiles for identity sides) and of every psi block read as Y^T.
  // Operator addresses are absolute (the task list is launched with x/z bases 0).
  void build_tc(const std::vector<ChainEntry, NoInitAlloc<ChainEntry>> &xs, const std::vector<ChainGroup> &vt,
                cudaStream_t s) {
    TcPlan P;
    plan_tc(xs, vt, P, nullptr, ops32 ? 4 : 8, tc_tiny);
    std::vector<TcEntry> &te = P.te;
    std::vector<TcGroup> &tg = P.tg;
    std::vector<TileSpec> &ts = P.ts;
    std::vector<PsiTileSpec> &ps = P.ps;
    const uint64_t opbytes = P.opbytes, psibytes = P.psibytes;
    for (int sh = 0; sh < 3; ++sh) ntc_shape[sh] = P.ntc_shape[sh];
    ntc = (int)tg.size();
    npts = (int)ps.size();
    if (ntc == 0) return;
    te.resize(te.size() + kTcChunkCopy, TcEntry{});  // the kernel's fixed-size descriptor chunks read past the end
    tce.upload(te, s);
    tcg.upload(tg, s);
    pts.upload(ps, s);
    optiles.alloc((size_t)opbytes);
    psitiles.alloc((size_t)psibytes);
    tc_counter.alloc(3);
    DBuf<TileSpec> tsd;
    tsd.upload(ts, s);
    CK(launch_build_tiles(tsd.p, (int)ts.size(), optiles.p, !ops32, s));
    CK(cudaStreamSynchronize(s));  // tsd is released on return
  }

  // device memory of the task list back to the allocator
  void release() {
    ent.release();
    xent.release();
    all.release();
    big.release();
    flat.release();
    red.release();
    scratch.release();
    tce.release();
    tcg.release();
    pts.release();
    optiles.release();
    psitiles.release();
    tc_counter.release();
    nall = nbig = nflat = ntc = ntiles = nred = npts = 0;
    ntc_shape[0] = ntc_shape[1] = ntc_shape[2] = 0;
    nent = red_total = scratch_n = 0;
  }

  void launch_tc(uint64_t yb, uint64_t tb, int *status, cudaStream_t s) const {
    if (ntc == 0) return;
    if (!status) throw Fail{DMRG_EINVAL, "tensor-core task list launched without a status word"};
    CK(launch_psi_tiles(pts.p, npts, reinterpret_cast<const double *>(yb), psitiles.p, s));
    int first = 0;
    for (int sh : {2, 1, 0}) {
      CK(launch_chain_tc2(tce.p, tcg.p + first, ntc_shape[sh], optiles.p, psitiles.p, tb, tc_counter.p + sh,
                          status, sh, s));
      first += ntc_shape[sh];
    }
  }

  // The launch sequence.  The chunk partials of a split task list go to the
  // list's own scratch array, or to ext (at least scratch_n doubles, cleared
  // here) when the caller provides one; nothing is allocated here.
  void launch(uint64_t xb, uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s, int *status = nullptr,
              double *ext = nullptr) const {
    double *part = ext ? ext : scratch.p;
    const uint64_t tb = split ? (uint64_t)(uintptr_t)part : db;
    if (split && scratch_n > 0) CK(cudaMemsetAsync(part, 0, scratch_n * sizeof(double), s));
    if (ops32) {
      CK(launch_chain_f32ops(xent.p, big.p, nbig, ntiles, xb, yb, zb, tb, s));
      CK(launch_chain_flat_f32ops(xent.p, flat.p, nflat, xb, yb, zb, tb, s, flat_wide ? 12 : 8));
    } else {
      CK(launch_chain_fp64(xent.p, big.p, nbig, ntiles, xb, yb, zb, tb, s));
      CK(launch_chain_flat_fp64(xent.p, flat.p, nflat, xb, yb, zb, tb, s, flat_wide ? 6 : 4));
    }
    launch_tc(yb, tb, status, s);
    if (split) CK(launch_reduce_partials(red.p, nred, red_total, part, (double *)(uintptr_t)db, s));
  }
};

static double entry_flops(int m, int n, int p, int q, bool xid, bool zid) {
  if (xid && zid) return 0.0;
  if (xid) return 2.0 * n * p * q;
  if (zid) return 2.0 * m * n * p;
  return 2.0 * std::min((double)m * n * p + (double)m * p * q, (double)n * p * q + (double)m * n * q);
}

// ---------------------------------------------------------------- temporaries

struct DevTemps {
  TempSet set;
  DBuf<double> arena[2];
  DBuf<double> coefs;
  DBuf<LincombTask> tasks;
};

// Materialize the temporaries of a TempSet (Sec. 2.2.3 pre-summation).
static void build_temps(DevTemps &T, const BlockLayout *lay[2], const double *stored[2],
                        cudaStream_t s) {
  T.set.layout(lay);
  for (int side = 0; side < 2; ++side) T.arena[side].alloc((size_t)std::max<int64_t>(T.set.total[side], 1));
  std::vector<double> coef;
  std::vector<int64_t> coef_off;
  std::vector<std::pair<int, int>> fam_list;
  for (int side = 0; side < 2; ++side)
    for (int f = 0; f < (int)T.set.fam[side].size(); ++f) {
      const TempFamily &TF = T.set.fam[side][f];
      const Family &SF = lay[side]->fam[TF.src_fam];
      coef_off.push_back((int64_t)coef.size());
      fam_list.push_back({side, f});
      const size_t base = coef.size();
      coef.resize(base + (size_t)TF.K() * SF.K(), 0.0);
      for (int t = 0; t < TF.K(); ++t)
        for (auto &u : TF.coefs[t]) coef[base + (size_t)t * SF.K() + u.first] += u.second;
    }
  T.coefs.upload(coef, s);
  std::vector<LincombTask> tasks;
  int ntiles = 0;
  for (size_t fi = 0; fi < fam_list.size(); ++fi) {
    const int side = fam_list[fi].first, f = fam_list[fi].second;
    const TempFamily &TF = T.set.fam[side][f];
    const BlockLayout &b = *lay[side];
    const Family &SF = b.fam[TF.src_fam];
    for (int a = 0; a < (int)b.sec.size(); ++a) {
      const int a2 = TF.bra[a];
      if (a2 < 0) continue;
      LincombTask t;
      t.out = eaddr(T.arena[side].p) + TF.base + TF.off[a];
      int64_t src;
      if (!TF.tr) {
        if (SF.off[a] < 0) continue;
        src = SF.base + SF.off[a];
      } else {
        if (SF.off[a2] < 0 || SF.bra[a2] != a) continue;
        src = SF.base + SF.off[a2];
      }
      t.src = eaddr(stored[side]) + src;
      t.coef = eaddr(T.coefs.p) + coef_off[fi];
      t.kout = TF.K();
      t.ksrc = SF.K();
      t.rows = b.sec[a2].dim;
      t.cols = b.sec[a].dim;
      t.tr = TF.tr ? 1 : 0;
      t.tile0 = ntiles;
      const int64_t E = (int64_t)t.rows * t.cols;
      ntiles += ((t.kout + 31) / 32) * (int)((E + 31) / 32);
      tasks.push_back(t);
    }
  }
  // temp slabs without a source slab stay zero
  for (int side = 0; side < 2; ++side)
    if (T.set.total[side] > 0)
      CK(cudaMemsetAsync(T.arena[side].p, 0, T.set.total[side] * sizeof(double), s));
  T.tasks.upload(tasks, s);
  CK(launch_lincomb_fp64(T.tasks.p, (int)tasks.size(), ntiles, s));
}

// ---------------------------------------------------------------- H.psi plan

struct RPiece {
  Ref l, r;
  Piece p;
};

struct HPlan {
  std::vector<RPiece> rps;  // resolved pieces of H at this position
  bool valid = false;
  int k = -1;
  const DevBlock *lb = nullptr, *rb = nullptr;
  Psi psi;
  DevTemps temps;
  DevChain chain;
  double flops = 0.0;
  long long ntasks = 0;
  DBuf<double> diag;
  // mixed precision: FP32 copies of the operators and temporaries + their task list
  bool lowp = false;
  DBuf<float> f32[4];  // left ops, right ops, left temps, right temps
  DevChain chain32;
};

}  // namespace dmrg

struct dmrg_ctx {
  int L = 0, N = 0, nu = 0, nd = 0, M = 0, prec = 0;
  int M_bwd = 0;  // kept states of right blocks (backward renormalizations); M for left blocks
  cudaStream_t stream = nullptr;
  dmrg::Integrals I;
  std::vector<std::unique_ptr<dmrg::DevBlock>> left, right;  // by size
  int k = 0, dir = 1;
  dmrg::HPlan plan;
  // wave function at the current position
  dmrg::DBuf<double> psi;
  bool psi_valid = false;
  // Davidson workspace
  dmrg::DBuf<double> V, AV, work, partial, small, r, t, hx;
  cusolverDnHandle_t solver = nullptr;
  dmrg::DBuf<double> sol_work;
  dmrg::DBuf<int> sol_info;
  // statistics: CUDA events around every H.psi kernel launch on the context stream
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  double hpsi_ms_folded = 0.0;
  long long hpsi_calls = 0;
  double hpsi_flops_acc = 0.0;
  long long dav_iters = 0;
  long long launch_base = 0;
  double last_resid = 0.0;
  long long dav_iters_lowp = 0;
  dmrg::DBuf<int> dstatus;  // set by bounded device waits that ran out
  dmrg::ChainTune tune;     // launch shape of H.psi task lists (dmrg_autotune)
  // density-matrix truncations: gap at the cut of the last one, smallest gap,
  // count, and how many had a near-degenerate cluster across the cut
  int refine_keep = 0;       // Ritz vectors carried between refinement steps (dmrg_set_davidson)
  int sweep_max_iter = 200;  // matvec cap of each Davidson step of a sweep
  int renorm_prec = DMRG_PREC_FP64;  // renormalization products: FP64 or FP32 O (dmrg_set_renorm_precision)
  long long plan_gen = 0;  // count of H.psi plan builds and releases (a batch's record of its members)
  double cut_gap = std::numeric_limits<double>::infinity();
  double min_cut_gap = std::numeric_limits<double>::infinity();
  long long truncations = 0, straddled = 0;
};

namespace dmrg {

static DevBlock *lblock(dmrg_ctx *c) {
  return c->k < (int)c->left.size() ? c->left[c->k].get() : nullptr;
}
static DevBlock *rblock(dmrg_ctx *c) {
  const int n = c->L - c->k - 2;
  return (n >= 0 && n < (int)c->right.size()) ? c->right[n].get() : nullptr;
}

static void require_blocks(dmrg_ctx *c) {
  if (!lblock(c) || !rblock(c))
    throw Fail{DMRG_ESTATE, "blocks for position " + std::to_string(c->k) + " are not built"};
}

static std::unique_ptr<DevBlock> empty_block(int side, int L) {
  auto b = std::make_unique<DevBlock>();
  build_layout(b->lay, side, L, {}, {{0, 0, 1}});
  return b;
}

// Resolve the (compressed) pieces of H at position k onto the two blocks;
// pieces on operators that vanish there are dropped.
static std::vector<RPiece> resolve_pieces(const Integrals &I, int k, const BlockLayout &L,
                                          const BlockLayout &R, TempSet &temps) {
  auto pieces = compress_pieces(hamiltonian_pieces(I, k, L.empty(), R.empty()));
  // linear-combination operators prepared in parallel, then numbered in piece order
  std::vector<PreparedTemp> pl(pieces.size()), pr(pieces.size());
  const size_t CH = 64;
  parallel_for((pieces.size() + CH - 1) / CH, [&](size_t c) {
    for (size_t i = c * CH; i < std::min(pieces.size(), (c + 1) * CH); ++i) {
      if (pieces[i].l.type == 2) pl[i] = prepare_temp(L, pieces[i].l);
      if (pieces[i].r.type == 2) pr[i] = prepare_temp(R, pieces[i].r);
    }
  });
  std::vector<RPiece> out;
  for (size_t i = 0; i < pieces.size(); ++i) {
    Piece &p = pieces[i];
    bool zl, zr;
    Ref l = p.l.type == 2 ? temps.make_prepared(0, L, p.l, std::move(pl[i]), zl) : resolve(p.l, 0, L, temps, zl);
    if (zl) continue;
    Ref r = p.r.type == 2 ? temps.make_prepared(1, R, p.r, std::move(pr[i]), zr) : resolve(p.r, 1, R, temps, zr);
    if (zr) continue;
    out.push_back({l, r, std::move(p)});
  }
  return out;
}

// Expand pieces over the psi blocks of Eq. wf_sec into the H.psi task list
// (Sec. 2.2.1): one entry per (piece, s -> s'), plus the transposed entry of
// Hermitian-conjugate pieces.  Returns the algorithmic FLOPs.  This part: the
// pieces [r0, r1); emit(output block, entry) receives the entries in build
// order.  Per piece, the site images of the four site states and the effective
// block of every block sector are tabulated once for all psi blocks.
template <class Emit>
static double expand_range(const std::vector<RPiece> &rps, size_t r0, size_t r1, const Arenas &A, const Psi &Y,
                           const BlockLayout &lb, Emit &&emit) {
  struct Eff {
    bool ok;
    int a2, rs, cs;
    uint64_t addr;
  };
  std::vector<Eff> effl((size_t)Y.nl), effr((size_t)Y.nr);
  double flops = 0.0;
  for (size_t ri = r0; ri < r1; ++ri) {
    const RPiece &rp = rps[ri];
    const Piece &p = rp.p;
    const int psl = mat_parity(p.sl), psr = mat_parity(p.sr);
    int b2[4], c2[4];
    double vb[4], vc[4];
    bool any_b = false, any_c = false;
    for (int x = 0; x < 4; ++x) {
      b2[x] = site_image(p.sl, x, vb[x]);
      c2[x] = site_image(p.sr, x, vc[x]);
      any_b |= b2[x] >= 0;
      any_c |= c2[x] >= 0;
    }
    if (!any_b || !any_c) continue;
    for (int x = 0; x < Y.nl; ++x) {
      Eff &E = effl[(size_t)x];
      E.ok = eff_block(rp.l, A, 0, x, E.a2, E.addr, E.rs, E.cs);
    }
    for (int x = 0; x < Y.nr; ++x) {
      Eff &E = effr[(size_t)x];
      E.ok = eff_block(rp.r, A, 1, x, E.a2, E.addr, E.rs, E.cs);
    }
    const bool xid = rp.l.arena < 0, zid = rp.r.arena < 0;
    for (size_t si = 0; si < Y.blk.size(); ++si) {
      const PsiBlock &s = Y.blk[si];
      const int sb = b2[s.b], sc = c2[s.c];
      if (sb < 0 || sc < 0) continue;
      const Eff &El = effl[(size_t)s.a];
      if (!El.ok) continue;
      const Eff &Er = effr[(size_t)s.d];
      if (!Er.ok) continue;
      const int so = Y.find(El.a2, sb, sc, Er.a2);
      if (so < 0) continue;
      const PsiBlock &t = Y.blk[so];
      const int na = npart(lb.sec[s.a]), nb = nsite(s.b), nc = nsite(s.c);
      const int sgn_exp = rp.r.par * (na + nb + nc) + psr * (na + nb) + psl * na;
      const double f = p.coef * vb[s.b] * vc[s.c] * ((sgn_exp & 1) ? -1.0 : 1.0);
      ChainEntry e{};
      e.x = El.addr;
      e.xrs = El.rs;
      e.xcs = El.cs;
      e.y = (uint64_t)s.off;
      e.yrs = s.md;
      e.ycs = 1;
      e.z = Er.addr;
      e.zrs = Er.cs;  // Z = R^T
      e.zcs = Er.rs;
      e.n = s.ma;
      e.p = s.md;
      e.f = f;
      emit(so, e);
      flops += entry_flops(t.ma, s.ma, s.md, t.md, xid, zid);
      if (p.hc) {
        ChainEntry h{};
        h.x = El.addr;
        h.xrs = El.cs;  // X = L^T
        h.xcs = El.rs;
        h.y = (uint64_t)t.off;
        h.yrs = t.md;
        h.ycs = 1;
        h.z = Er.addr;  // Z = R
        h.zrs = Er.rs;
        h.zcs = Er.cs;
        h.n = t.ma;
        h.p = t.md;
        h.f = f;
        emit((int)si, h);
        flops += entry_flops(s.ma, t.ma, t.md, s.md, xid, zid);
      }
    }
  }
  return flops;
}

// The pieces are cut into a fixed number of ranges (independent of the host's
// core count) that worker threads expand; ranges keep piece order, so the
// result is that of a sequential expansion and the FLOP sum (exact integers)
// is identical.
static size_t expand_ranges(const std::vector<RPiece> &rps) { return std::min<size_t>(rps.size(), 64); }

// The task list in build order (per-range parts, grouped later by finish()).
static void expand_hpsi(const std::vector<RPiece> &rps, const Arenas &A, const Psi &Y,
                        const BlockLayout &lb, ChainList &CL, double &flops) {
  const size_t nr = expand_ranges(rps);
  std::vector<ChainList::Keyed> part(nr);
  std::vector<double> fl(nr, 0.0);
  parallel_for(nr, [&](size_t c) {
    ChainList::Keyed &out = part[c];
    fl[c] = expand_range(rps, c * rps.size() / nr, (c + 1) * rps.size() / nr, A, Y, lb,
                         [&](int key, const ChainEntry &e) { out.push_back({key, e}); });
  });
  flops = 0.0;
  for (size_t c = 0; c < nr; ++c) {
    CL.parts.push_back(std::move(part[c]));
    flops += fl[c];
  }
}

static std::vector<ChainGroup> psi_protos(const Psi &Y);

// The task list grouped by output block, as finish() would leave it, built in
// two passes over the pieces: count the entries of every (range, output block),
// then write each entry straight to its place (no intermediate list).
static void expand_hpsi_grouped(const std::vector<RPiece> &rps, const Arenas &A, const Psi &Y,
                                const BlockLayout &lb, ChainList &CL, double &flops) {
  const size_t nr = expand_ranges(rps), ng = Y.blk.size();
  std::vector<int64_t> cnt(nr * ng, 0);
  std::vector<double> fl(nr, 0.0);
  parallel_for(nr, [&](size_t c) {
    int64_t *k = cnt.data() + c * ng;
    fl[c] = expand_range(rps, c * rps.size() / nr, (c + 1) * rps.size() / nr, A, Y, lb,
                         [&](int key, const ChainEntry &) { ++k[(size_t)key]; });
  });
  std::vector<int64_t> start(ng + 1, 0), off(nr * ng);
  int64_t run = 0;
  for (size_t g = 0; g < ng; ++g) {
    start[g] = run;
    for (size_t c = 0; c < nr; ++c) {
      off[c * ng + g] = run;
      run += cnt[c * ng + g];
    }
  }
  start[ng] = run;
  CL.flat.clear();
  CL.flat.resize((size_t)run);  // every element is written by the second pass
  parallel_for(nr, [&](size_t c) {
    int64_t *o = off.data() + c * ng;
    ChainEntry *dst = CL.flat.data();
    expand_range(rps, c * rps.size() / nr, (c + 1) * rps.size() / nr, A, Y, lb,
                 [&](int key, const ChainEntry &e) { dst[o[(size_t)key]++] = e; });
  });
  flops = 0.0;
  for (size_t c = 0; c < nr; ++c) flops += fl[c];
  const std::vector<ChainGroup> protos = psi_protos(Y);
  CL.grp.clear();
  CL.ntiles = 0;
  for (size_t g = 0; g < ng; ++g) {
    const int64_t n = start[g + 1] - start[g];
    if (n == 0) continue;
    ChainGroup G = protos[g];
    G.first = (int)start[g];
    G.count = (int)n;
    G.tile0 = CL.ntiles;
    CL.ntiles += ((G.m + 31) / 32) * ((G.q + 31) / 32);
    CL.grp.push_back(G);
  }
}

static std::vector<ChainGroup> psi_protos(const Psi &Y) {
  std::vector<ChainGroup> protos(Y.blk.size());
  for (size_t i = 0; i < Y.blk.size(); ++i) {
    ChainGroup g{};
    g.d = (uint64_t)Y.blk[i].off;
    g.drs = Y.blk[i].md;
    g.dcs = 1;
    g.m = Y.blk[i].ma;
    g.q = Y.blk[i].md;
    protos[i] = g;
  }
  return protos;
}

// The H.psi task list of the current plan over the FP64 masters or the FP32
// copies (mixed precision), grouped by output psi block.
static void hpsi_chainlist(dmrg_ctx *c, bool f32, ChainList &CL, double &flops) {
  HPlan &P = c->plan;
  DevBlock *lb = lblock(c), *rb = rblock(c);
  if (f32) {
    Arenas A32{{&lb->lay, &rb->lay}, {P.f32[0].p, P.f32[1].p}, &P.temps.set, {P.f32[2].p, P.f32[3].p}, 4};
    expand_hpsi_grouped(P.rps, A32, P.psi, lb->lay, CL, flops);
  } else {
    Arenas A{{&lb->lay, &rb->lay}, {lb->arena(), rb->arena()}, &P.temps.set,
             {P.temps.arena[0].p, P.temps.arena[1].p}, 8};
    expand_hpsi_grouped(P.rps, A, P.psi, lb->lay, CL, flops);
  }
}

static void build_hplan(dmrg_ctx *c) {
  HPlan &P = c->plan;
  require_blocks(c);
  DevBlock *lb = lblock(c), *rb = rblock(c);
  if (P.valid && P.k == c->k && P.lb == lb && P.rb == rb) return;
  P.valid = false;
  ++c->plan_gen;
  P.k = c->k;
  P.lb = lb;
  P.rb = rb;
  P.psi = psi_layout(lb->lay, rb->lay, c->nu, c->nd);
  const Psi &Y = P.psi;
  P.temps.set = TempSet();
  P.rps = resolve_pieces(c->I, c->k, lb->lay, rb->lay, P.temps.set);
  const BlockLayout *lay[2] = {&lb->lay, &rb->lay};
  const double *stored[2] = {lb->arena(), rb->arena()};
  build_temps(P.temps, lay, stored, c->stream);
  {
    ChainList CL;
    double flops = 0.0;
    hpsi_chainlist(c, false, CL, flops);
    P.chain.upload(CL, c->stream, false, true, c->tune);
    P.flops = flops;
    P.ntasks = (long long)CL.flat.size();
    CK(cudaStreamSynchronize(c->stream));  // host vectors are released at the end of the scope
  }
  P.diag.alloc((size_t)std::max<int64_t>(Y.dim, 1));
  CK(cudaMemsetAsync(P.diag.p, 0, Y.dim * sizeof(double), c->stream));
  CK(launch_diag_fp64(P.chain.ent.p, P.chain.all.p, P.chain.nall, 0, 0, P.diag.p, c->stream));
  P.lowp = c->prec != DMRG_PREC_FP64;
  if (c->prec == DMRG_PREC_FP32) {
    // FP32 working copies of every operand of the H.psi task list (Davidson matvecs)
    const double *src[4] = {lb->arena(), rb->arena(), P.temps.arena[0].p, P.temps.arena[1].p};
    const int64_t cnt[4] = {lb->lay.total, rb->lay.total, P.temps.set.total[0], P.temps.set.total[1]};
    for (int i = 0; i < 4; ++i) {
      P.f32[i].alloc((size_t)std::max<int64_t>(cnt[i], 1));
      if (cnt[i] > 0 && src[i]) CK(launch_to_f32(P.f32[i].p, src[i], cnt[i], c->stream));
    }
    ChainList CL32;
    double fl32 = 0.0;
    hpsi_chainlist(c, true, CL32, fl32);
    P.chain32.upload(CL32, c->stream, false, true, c->tune, true);
    CK(cudaStreamSynchronize(c->stream));
  } else if (c->prec == DMRG_PREC_BF16X3) {
    // the tensor-core list reads the FP64 masters: tiles are split straight from them, and
    // blocks the tensor cores do not take run in FP64 (no FP32 copies are held)
    ChainList CLt;
    double flt = 0.0;
    hpsi_chainlist(c, false, CLt, flt);
    P.chain32.upload(CLt, c->stream, true, true, c->tune, false);
    CK(cudaStreamSynchronize(c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  P.valid = true;
}

// Report a bounded device-side wait that ran out (the kernel skipped its work).
static void check_status(dmrg_ctx *c) {
  int st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(st, c->dstatus.p, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st[0]) {
    CK(cudaMemsetAsync(c->dstatus.p, 0, sizeof(st), c->stream));
    std::string where;
    for (int i = 1; i < 8; ++i) where += (i > 1 ? "," : "") + std::to_string(st[i]);
    throw Fail{DMRG_ETIMEOUT, "a tensor-core completion wait ran out; results of that call are invalid "
                              "(site,parity,block,aux0,aux1,bar_lo,bar_hi = " + where + ")"};
  }
}

static void fold_events(dmrg_ctx *c) {
  if (c->ev_used == 0) return;
  CK(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    c->hpsi_ms_folded += ms;
  }
  c->ev_used = 0;
}

static void hpsi_dev(dmrg_ctx *c, const double *psi, double *sigma, bool fp64 = false) {
  HPlan &P = c->plan;
  const bool lowp = P.lowp && !fp64;
  CK(cudaMemsetAsync(sigma, 0, P.psi.dim * sizeof(double), c->stream));
  if (c->ev_used + 2 > 4096) fold_events(c);
  while (c->ev.size() < c->ev_used + 2) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  CK(cudaEventRecord(c->ev[c->ev_used], c->stream));
  (lowp ? P.chain32 : P.chain).launch(0, (uint64_t)(uintptr_t)psi, 0, (uint64_t)(uintptr_t)sigma, c->stream,
                                      c->dstatus.p);
  CK(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
  c->ev_used += 2;
  c->hpsi_calls += 1;
  c->hpsi_flops_acc += P.flops;
}

// ---------------------------------------------------------------- renormalization

// Operators of the new block: O^T (sum_pieces blk (x) site) O per new sector
// pair (Sec. 2.2.2, Eq. renorm_mat), never forming the enlarged matrices.
static std::unique_ptr<DevBlock> renormalize_block(dmrg_ctx *c, int direction, const Enlarged &enl,
                                                   const std::vector<int> &kept,
                                                   DBuf<double> &Odev,
                                                   const std::vector<int64_t> &Ooff) {
  const int side = direction > 0 ? 0 : 1;
  DevBlock *old = side == 0 ? lblock(c) : rblock(c);
  auto nb = std::make_unique<DevBlock>();
  std::vector<Sector> sec;
  std::vector<int> new_of_enl(enl.size(), -1);
  for (size_t e = 0; e < enl.size(); ++e)
    if (kept[e] > 0) {
      new_of_enl[e] = (int)sec.size();
      sec.push_back({enl[e].nu, enl[e].nd, kept[e]});
    }
  if (sec.empty()) throw Fail{DMRG_EINVAL, "renormalization keeps no state"};
  std::vector<int> sites;
  if (side == 0) for (int s = 0; s <= c->k; ++s) sites.push_back(s);
  else for (int s = c->k + 1; s < c->L; ++s) sites.push_back(s);
  build_layout(nb->lay, side, c->L, sites, sec);
  nb->ops.alloc((size_t)std::max<int64_t>(nb->lay.total, 1));
  CK(cudaMemsetAsync(nb->ops.p, 0, std::max<int64_t>(nb->lay.total, 1) * sizeof(double), c->stream));

  auto defs = new_block_ops(c->I, c->k, side, nb->lay, old->lay.empty());
  DevTemps temps;
  struct RD {
    int fam, k;
    Ref blk;
    Mat4 site;
    double coef;
  };
  std::vector<RD> rds;
  for (auto &d : defs)
    for (auto &hp : d.def) {
      bool z;
      Ref r = resolve(hp.blk, side, old->lay, temps.set, z);
      if (z) continue;
      rds.push_back({d.fam, d.k, r, hp.site, hp.coef});
    }
  const BlockLayout *lay[2];
  const double *stored[2];
  lay[side] = &old->lay;
  stored[side] = old->arena();
  // the other side has no temporaries; give it a harmless layout
  BlockLayout dummy;
  build_layout(dummy, 1 - side, c->L, {}, {{0, 0, 1}});
  lay[1 - side] = &dummy;
  stored[1 - side] = nullptr;
  build_temps(temps, lay, stored, c->stream);
  Arenas A{{lay[0], lay[1]}, {stored[0], stored[1]}, &temps.set,
           {temps.arena[0].p, temps.arena[1].p}, 8};

  // sub-block lookup: enlarged sector index + row offset of (block sector, site
  // state), a dense table over the old block's sectors and the four site states
  const int nob = (int)old->lay.sec.size();
  std::vector<std::pair<int, int>> where((size_t)nob * 4, {-1, 0});
  for (size_t e = 0; e < enl.size(); ++e)
    for (auto &sb : enl[e].sub) {
      const int bs = side == 0 ? sb.x : sb.y, st = side == 0 ? sb.y : sb.x;
      where[(size_t)bs * 4 + st] = {(int)e, sb.roff};
    }

  // output groups: (family, k, new ket sector), numbered in order of first use
  const int nns = (int)nb->lay.sec.size();
  std::vector<int64_t> fam_gbase(nb->lay.fam.size() + 1, 0);
  for (size_t f = 0; f < nb->lay.fam.size(); ++f)
    fam_gbase[f + 1] = fam_gbase[f] + (int64_t)nb->lay.fam[f].K() * nns;
  std::vector<int> gid((size_t)fam_gbase.back(), -1);
  std::vector<ChainGroup> protos;
  ChainList CL;
  const double *Op = Odev.p;
  for (auto &rd : rds) {
    const Family &F = nb->lay.fam[rd.fam];
    const int pblk = rd.blk.par, psite = mat_parity(rd.site);
    for (size_t e = 0; e < enl.size(); ++e) {
      const int An = new_of_enl[e];
      if (An < 0) continue;
      const int Bn = F.bra[An];
      if (Bn < 0) continue;
      for (auto &sb : enl[e].sub) {
        // ket sub-block (x, y): left (a, b), right (c, d)
        const int blk_sec = side == 0 ? sb.x : sb.y;
        const int site_st = side == 0 ? sb.y : sb.x;
        double sv;
        const int site2 = site_image(rd.site, site_st, sv);
        if (site2 < 0) continue;
        int b2, rs, cs;
        uint64_t addr;
        if (!eff_block(rd.blk, A, side, blk_sec, b2, addr, rs, cs)) continue;
        const std::pair<int, int> &w2 = where[(size_t)b2 * 4 + site2];
        if (w2.first < 0) continue;
        const int e2 = w2.first, roff2 = w2.second;
        if (new_of_enl[e2] != Bn) continue;
        const int sgn_exp = side == 0 ? psite * npart(old->lay.sec[blk_sec])
                                      : pblk * nsite(site_st);
        const double f = rd.coef * sv * ((sgn_exp & 1) ? -1.0 : 1.0);
        const int mk = kept[e], mk2 = kept[e2];
        const int mb = old->lay.sec[blk_sec].dim, mb2 = old->lay.sec[b2].dim;
        int &gi = gid[(size_t)(fam_gbase[rd.fam] + (int64_t)rd.k * nns + An)];
        if (gi < 0) {
          ChainGroup cg{};
          cg.d = eaddr(nb->ops.p) + F.base + F.off[An] + (int64_t)rd.k * mk2 * mk;
          cg.drs = mk;
          cg.dcs = 1;
          cg.m = mk2;
          cg.q = mk;
          gi = (int)protos.size();
          protos.push_back(cg);
        }
        ChainEntry ce{};
        // X = O_{e2}[rows of (b2, site2)]^T : mk2 x mb2
        ce.x = eaddr(Op) + Ooff[e2] + (int64_t)roff2 * mk2;
        ce.xrs = 1;
        ce.xcs = mk2;
        ce.y = addr;
        ce.yrs = rs;
        ce.ycs = cs;
        // Z = O_e[rows of (x, y)] : mb x mk
        ce.z = eaddr(Op) + Ooff[e] + (int64_t)sb.roff * mk;
        ce.zrs = mk;
        ce.zcs = 1;
        ce.n = mb2;
        ce.p = mb;
        ce.f = f;
        if (rd.blk.arena < 0) {  // identity block operator: n == p
          ce.y = ~0ull;
          ce.n = mb;
        }
        CL.ent.push_back({gi, ce});
      }
    }
  }
  CL.finish(protos);
  DevChain dc;
  if (c->renorm_prec == DMRG_PREC_FP32) {
    // FP32 products: O (both X = O^T and Z = O) rounded to FP32, the old block's
    // operators converted to FP32 as the kernel reads them, FP32 accumulation per
    // output block, FP64 result
    DBuf<float> O32;
    const int64_t nO = (int64_t)Odev.n;
    O32.alloc((size_t)std::max<int64_t>(nO, 1));
    if (nO > 0) CK(launch_to_f32(O32.p, Odev.p, nO, c->stream));
    const uint64_t d64 = eaddr(Op), f32b = (uint64_t)(uintptr_t)O32.p / 4;
    for (auto &ce : CL.flat) {
      ce.x = f32b + (ce.x - d64);
      ce.z = f32b + (ce.z - d64);
    }
    dc.upload(CL, c->stream, false, false, ChainTune(), true);
    dc.launch(0, 0, 0, 0, c->stream);
    CK(cudaStreamSynchronize(c->stream));
  } else {
    dc.upload(CL, c->stream);
    dc.launch(0, 0, 0, 0, c->stream);
    CK(cudaStreamSynchronize(c->stream));
  }
  nb->parent = enl;
  nb->kept = kept;
  nb->Ooff = Ooff;
  std::swap(nb->O.p, Odev.p);
  std::swap(nb->O.n, Odev.n);
  return nb;
}

// ---------------------------------------------------------------- RDM + truncation

static void rdm_truncate(dmrg_ctx *c, int direction, const Enlarged &enl, std::vector<int> &kept,
                         DBuf<double> &Odev, std::vector<int64_t> &Ooff, double &dw) {
  HPlan &P = c->plan;
  const Psi &Y = P.psi;
  const int ne = (int)enl.size();
  std::vector<int64_t> roff(ne);
  int64_t tot = 0;
  for (int e = 0; e < ne; ++e) {
    roff[e] = tot;
    tot += (int64_t)enl[e].dim * enl[e].dim;
  }
  DBuf<double> rho;
  rho.alloc((size_t)std::max<int64_t>(tot, 1));
  CK(cudaMemsetAsync(rho.p, 0, std::max<int64_t>(tot, 1) * sizeof(double), c->stream));
  // rho^L[(a,b),(a',b')] = sum_{c,d} psi_abcd psi_a'b'cd^T ; rho^R[(c,d),(c',d')] = sum_{a,b} psi_abcd^T psi_abc'd'
  std::map<std::pair<int, int>, std::pair<int, int>> where;
  for (int e = 0; e < ne; ++e)
    for (auto &sb : enl[e].sub) where[{sb.x, sb.y}] = {e, sb.roff};
  std::vector<ChainGroup> protos;
  std::map<std::tuple<int, int, int, int>, int> gid;
  ChainList CL;
  for (auto &s1 : Y.blk)
    for (auto &s2 : Y.blk) {
      std::pair<int, int> k1, k2;
      if (direction > 0) {
        if (s1.c != s2.c || s1.d != s2.d) continue;
        k1 = {s1.a, s1.b};
        k2 = {s2.a, s2.b};
      } else {
        if (s1.a != s2.a || s1.b != s2.b) continue;
        k1 = {s1.c, s1.d};
        k2 = {s2.c, s2.d};
      }
      auto w1 = where.at(k1), w2 = where.at(k2);
      if (w1.first != w2.first) continue;
      const int e = w1.first, n = enl[e].dim;
      auto key = std::make_tuple(k1.first, k1.second, k2.first, k2.second);
      int gi;
      auto git = gid.find(key);
      const int rows = direction > 0 ? s1.ma : s1.md;
      const int cols = direction > 0 ? s2.ma : s2.md;
      if (git == gid.end()) {
        ChainGroup g{};
        g.d = eaddr(rho.p) + roff[e] + (int64_t)w1.second * n + w2.second;
        g.drs = n;
        g.dcs = 1;
        g.m = rows;
        g.q = cols;
        gi = (int)protos.size();
        protos.push_back(g);
        gid[key] = gi;
      } else {
        gi = git->second;
      }
      ChainEntry ce{};
      ce.x = ~0ull;
      if (direction > 0) {  // psi1 (ma x md) * psi2^T (md x ma')
        ce.y = (uint64_t)s1.off;
        ce.yrs = s1.md;
        ce.ycs = 1;
        ce.z = (uint64_t)s2.off;
        ce.zrs = 1;
        ce.zcs = s2.md;
        ce.n = s1.ma;
        ce.p = s1.md;
      } else {  // psi1^T (md x ma) * psi2 (ma x md')
        ce.y = (uint64_t)s1.off;
        ce.yrs = 1;
        ce.ycs = s1.md;
        ce.z = (uint64_t)s2.off;
        ce.zrs = s2.md;
        ce.zcs = 1;
        ce.n = s1.md;
        ce.p = s1.ma;
      }
      ce.f = 1.0;
      CL.ent.push_back({gi, ce});
    }
  CL.finish(protos);
  DevChain dc;
  dc.upload(CL, c->stream);
  const uint64_t pb = (uint64_t)(uintptr_t)c->psi.p;
  dc.launch(0, pb, pb, 0, c->stream);

  // per-sector eigendecomposition (LAPACK-style syevd, eigenvalues ascending)
  int maxn = 0;
  for (auto &e : enl) maxn = std::max(maxn, e.dim);
  if (!c->solver) {
    CKS(cusolverDnCreate(&c->solver));
  }
  CKS(cusolverDnSetStream(c->solver, c->stream));
  int lwork = 0;
  CKS(cusolverDnDsyevd_bufferSize(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, maxn,
                                  rho.p, maxn, nullptr, &lwork));
  c->sol_work.alloc((size_t)std::max(lwork, 1));
  c->sol_info.alloc(1);
  std::vector<int64_t> eoff(ne);
  int64_t etot = 0;
  for (int e = 0; e < ne; ++e) {
    eoff[e] = etot;
    etot += enl[e].dim;
  }
  DBuf<double> ev;
  ev.alloc((size_t)std::max<int64_t>(etot, 1));
  for (int e = 0; e < ne; ++e) {
    const int n = enl[e].dim;
    if (n == 0) continue;
    CKS(cusolverDnDsyevd(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                         rho.p + roff[e], n, ev.p + eoff[e], c->sol_work.p, lwork, c->sol_info.p));
  }
  std::vector<double> evh(etot);
  CK(cudaMemcpyAsync(evh.data(), ev.p, etot * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // global top-M selection: descending eigenvalue, ties by (sector, in-sector order)
  std::vector<std::vector<double>> evs(ne);
  for (int e = 0; e < ne; ++e) evs[e].assign(evh.begin() + eoff[e], evh.begin() + eoff[e] + enl[e].dim);
  const int mkeep = direction > 0 ? c->M : c->M_bwd;  // kept states of the new left / right block
  KeptSet ks = choose_kept(evs, mkeep, 1e-13);
  kept = ks.kept;
  std::vector<std::vector<int>> &cols = ks.cols;
  dw = ks.trace - ks.kept_weight;
  c->cut_gap = ks.cut_gap;
  c->min_cut_gap = std::min(c->min_cut_gap, ks.cut_gap);
  c->truncations++;
  if (ks.cut_gap < kTruncCluster) c->straddled++;
  Ooff.assign(ne, 0);
  int64_t otot = 0;
  for (int e = 0; e < ne; ++e) {
    Ooff[e] = otot;
    otot += (int64_t)enl[e].dim * kept[e];
  }
  Odev.alloc((size_t)std::max<int64_t>(otot, 1));
  std::vector<int> allcols;
  std::vector<int64_t> coff(ne);
  for (int e = 0; e < ne; ++e) {
    coff[e] = (int64_t)allcols.size();
    allcols.insert(allcols.end(), cols[e].begin(), cols[e].end());
  }
  DBuf<int> dcols;
  dcols.upload(allcols, c->stream);
  for (int e = 0; e < ne; ++e)
    if (kept[e] > 0)
      CK(launch_gather_columns(Odev.p + Ooff[e], rho.p + roff[e], enl[e].dim, dcols.p + coff[e],
                               kept[e], c->stream));
  CK(cudaStreamSynchronize(c->stream));
}

// ---------------------------------------------------------------- wave-function prediction

// Forward move k -> k+1 (new left block built from O): psi'(A, c, e, f) =
// sum_{(a,b) in A, d} O_A[(a,b)]^T psi(a,b,c,d) O^R_d[(e,f)]^T, with O^R the
// renormalization that built the old right block.  Backward move is the mirror.
static void predict_psi(dmrg_ctx *c, const Psi &old, const DBuf<double> &oldpsi, int direction,
                        const DevBlock &nb) {
  c->psi_valid = false;
  DevBlock *lb = lblock(c), *rb = rblock(c);  // position already moved
  if (!lb || !rb) return;
  const int on = direction > 0 ? c->L - c->k - 1 : c->k + 1;
  const auto &store = direction > 0 ? c->right : c->left;
  const DevBlock *otherp = on < (int)store.size() ? store[on].get() : nullptr;
  if (!otherp) return;  // released by dmrg_release_block: no prediction
  const DevBlock &other = *otherp;
  // "other" is the block whose parent enlarged layout splits into the new site + new block
  if (other.parent.empty()) return;
  Psi Y = psi_layout(lb->lay, rb->lay, c->nu, c->nd);
  std::vector<ChainGroup> protos(Y.blk.size());
  for (size_t i = 0; i < Y.blk.size(); ++i) {
    ChainGroup g{};
    g.d = (uint64_t)Y.blk[i].off;
    g.drs = Y.blk[i].md;
    g.dcs = 1;
    g.m = Y.blk[i].ma;
    g.q = Y.blk[i].md;
    protos[i] = g;
  }
  // enlarged sector of the new block for each old (x, y) pair
  std::map<std::pair<int, int>, std::pair<int, int>> where_new;
  for (size_t e = 0; e < nb.parent.size(); ++e)
    for (auto &sb : nb.parent[e].sub) where_new[{sb.x, sb.y}] = {(int)e, sb.roff};
  std::vector<int> new_of_enl(nb.parent.size(), -1);
  for (size_t e = 0, n = 0; e < nb.parent.size(); ++e)
    if (nb.kept[e] > 0) new_of_enl[e] = (int)n++;
  std::vector<int> oth_of_enl(other.parent.size(), -1);
  for (size_t e = 0, n = 0; e < other.parent.size(); ++e)
    if (other.kept[e] > 0) oth_of_enl[e] = (int)n++;
  ChainList CL;
  for (auto &s : old.blk) {
    if (direction > 0) {
      // new-left sector from (a, b)
      auto wn = where_new.find({s.a, s.b});
      if (wn == where_new.end()) continue;
      const int eA = wn->second.first;
      const int A = new_of_enl[eA];
      if (A < 0) continue;
      // old right sector d expands into (e_site, f) sub-blocks of other.parent[enl of d]
      int ed = -1;
      for (size_t e = 0; e < other.parent.size(); ++e)
        if (oth_of_enl[e] == s.d) ed = (int)e;
      if (ed < 0) continue;
      const int mA = nb.kept[eA], md = other.kept[ed];
      for (auto &sb : other.parent[ed].sub) {
        const int so = Y.find(A, s.c, sb.x, sb.y);
        if (so < 0) continue;
        ChainEntry ce{};
        ce.x = eaddr(nb.O.p) + nb.Ooff[eA] + (int64_t)wn->second.second * mA;  // O_A rows^T
        ce.xrs = 1;
        ce.xcs = mA;
        ce.y = eaddr(oldpsi.p) + s.off;
        ce.yrs = s.md;
        ce.ycs = 1;
        ce.z = eaddr(other.O.p) + other.Ooff[ed] + (int64_t)sb.roff * md;  // (O^R_d rows)^T
        ce.zrs = 1;
        ce.zcs = md;
        ce.n = s.ma;
        ce.p = s.md;
        ce.f = 1.0;
        CL.ent.push_back({so, ce});
      }
    } else {
      auto wn = where_new.find({s.c, s.d});
      if (wn == where_new.end()) continue;
      const int eD = wn->second.first;
      const int D = new_of_enl[eD];
      if (D < 0) continue;
      int ea = -1;
      for (size_t e = 0; e < other.parent.size(); ++e)
        if (oth_of_enl[e] == s.a) ea = (int)e;
      if (ea < 0) continue;
      const int mD = nb.kept[eD], ma = other.kept[ea];
      for (auto &sb : other.parent[ea].sub) {
        const int so = Y.find(sb.x, sb.y, s.b, D);
        if (so < 0) continue;
        ChainEntry ce{};
        ce.x = eaddr(other.O.p) + other.Ooff[ea] + (int64_t)sb.roff * ma;  // O^L_a rows
        ce.xrs = ma;
        ce.xcs = 1;
        ce.y = eaddr(oldpsi.p) + s.off;
        ce.yrs = s.md;
        ce.ycs = 1;
        ce.z = eaddr(nb.O.p) + nb.Ooff[eD] + (int64_t)wn->second.second * mD;  // O_D rows
        ce.zrs = mD;
        ce.zcs = 1;
        ce.n = s.ma;
        ce.p = s.md;
        ce.f = 1.0;
        CL.ent.push_back({so, ce});
      }
    }
  }
  CL.finish(protos);
  c->psi.alloc((size_t)std::max<int64_t>(Y.dim, 1));
  CK(cudaMemsetAsync(c->psi.p, 0, Y.dim * sizeof(double), c->stream));
  DevChain dc;
  dc.upload(CL, c->stream);
  dc.launch(0, 0, 0, (uint64_t)(uintptr_t)c->psi.p, c->stream);
  CK(cudaStreamSynchronize(c->stream));
  c->psi_valid = !CL.flat.empty();
}

static void do_renormalize(dmrg_ctx *c, int direction, const int *kept_in, const double *O,
                           double *dw_out, int *kept_out) {
  if (O == nullptr) require_blocks(c);
  else if (!(direction > 0 ? lblock(c) : rblock(c)))
    throw Fail{DMRG_ESTATE, "the block to enlarge is not built"};
  if (direction > 0 && c->k >= c->L - 2) throw Fail{DMRG_ESTATE, "cannot move right of L-2"};
  if (direction < 0 && c->k <= 0) throw Fail{DMRG_ESTATE, "cannot move left of 0"};
  const int side = direction > 0 ? 0 : 1;
  DevBlock *old = side == 0 ? lblock(c) : rblock(c);
  Enlarged enl = enlarged(old->lay, direction);
  std::vector<int> kept;
  DBuf<double> Odev;
  std::vector<int64_t> Ooff;
  double dw = 0.0;
  if (O == nullptr) {
    build_hplan(c);
    if (!c->psi_valid) throw Fail{DMRG_ESTATE, "no wave function at this position (run dmrg_davidson)"};
    rdm_truncate(c, direction, enl, kept, Odev, Ooff, dw);
  } else {
    if (!kept_in) throw Fail{DMRG_EINVAL, "kept dims required with an explicit O"};
    kept.assign(kept_in, kept_in + enl.size());
    Ooff.assign(enl.size(), 0);
    int64_t tot = 0;
    for (size_t e = 0; e < enl.size(); ++e) {
      if (kept[e] < 0 || kept[e] > enl[e].dim) throw Fail{DMRG_EINVAL, "kept dim out of range"};
      Ooff[e] = tot;
      tot += (int64_t)enl[e].dim * kept[e];
    }
    Odev.alloc((size_t)std::max<int64_t>(tot, 1));
    if (tot) CK(cudaMemcpyAsync(Odev.p, O, tot * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  auto nb = renormalize_block(c, direction, enl, kept, Odev, Ooff);
  // keep the old psi for the prediction
  Psi oldlay = c->plan.valid ? c->plan.psi : Psi();
  DBuf<double> oldpsi;
  const bool can_predict = (O == nullptr) && c->psi_valid && c->plan.valid;
  if (can_predict) std::swap(oldpsi.p, c->psi.p), std::swap(oldpsi.n, c->psi.n);
  c->plan.valid = false;
  c->psi_valid = false;
  DevBlock *nbp = nb.get();
  if (side == 0) {
    if ((int)c->left.size() <= c->k + 1) c->left.resize(c->k + 2);
    c->left[c->k + 1] = std::move(nb);
    c->k += 1;
  } else {
    const int n = c->L - c->k - 1;
    if ((int)c->right.size() <= n) c->right.resize(n + 1);
    c->right[n] = std::move(nb);
    c->k -= 1;
  }
  c->dir = direction;
  if (can_predict) predict_psi(c, oldlay, oldpsi, direction, *nbp);
  if (dw_out) *dw_out = dw;
  if (kept_out) std::copy(kept.begin(), kept.end(), kept_out);
}

// ---------------------------------------------------------------- Davidson

// Relative size of the seeded admixture added to every Davidson start vector
// (see davidson_core).
static constexpr double kGuessAdmixture = 1e-3;

// One Davidson run (Sec. 2.2.1) from the current psi.  fp64: matvecs with the
// FP64 task list; otherwise the context's working precision.  floor: extra
// residual threshold (the attainable residual of low-precision matvecs).
static void davidson_core(dmrg_ctx *c, double tol, double floor_rel, int max_iter, bool fp64,
                          double *energy, int *iters, bool &conv) {
  build_hplan(c);
  HPlan &P = c->plan;
  const int64_t n = P.psi.dim;
  const int kmax = std::min<int64_t>(24, std::max<int64_t>(n, 1));
  c->V.alloc((size_t)kmax * n);
  c->AV.alloc((size_t)kmax * n);
  c->r.alloc(n);
  c->t.alloc(n);
  c->hx.alloc(n);
  c->partial.alloc((size_t)dots_partial_blocks(n) * 32);
  c->small.alloc(4096);
  double *G = c->small.p;              // kmax x kmax subspace matrix (row-major, ld 32)
  double *evals = c->small.p + 1024;   // 32
  double *evecs = c->small.p + 1056;   // up to 32 x 32
  double *dots = c->small.p + 2200;    // 32
  double *scal = c->small.p + 2300;    // theta, norm^2
  cudaStream_t s = c->stream;
  std::vector<double> Gh(32 * 32, 0.0);

  // start vector
  if (!c->psi_valid) {
    c->psi.alloc(n);
    CK(launch_fill_guess(c->psi.p, n, 12345ull, s));
  }
  CK(cudaMemcpyAsync(c->V.p, c->psi.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  auto normalize = [&](double *x) {
    CK(launch_dots(x, 1, n, x, c->partial.p, scal + 1, s));
    CK(launch_scale(x, scal + 1, 1, n, s));
  };
  normalize(c->V.p);
  if (n > 1) {
    // A start vector from the previous step lies in the symmetry subspace of
    // that step's state (H commutes with S^2 and with the spin flip), and an
    // FP64 Krylov space never leaves it: if the lowest state of this position
    // lies in another subspace, it would never be found.  A fixed seeded
    // admixture of relative size ~6e-4 restores a component along every
    // eigenvector, as in a Lanczos run from a random start.
    CK(launch_fill_guess(c->t.p, n, 0x5eedull, s));
    CK(launch_axpy(c->V.p, c->t.p, kGuessAdmixture / std::sqrt((double)n), n, s));
    normalize(c->V.p);
  }
  int k = 1;
  hpsi_dev(c, c->V.p, c->AV.p, fp64);
  // G[0][0]
  CK(launch_dots(c->V.p, 1, n, c->AV.p, c->partial.p, dots, s));
  CK(cudaMemcpyAsync(Gh.data(), dots, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double theta = Gh[0];
  int it = 0;
  conv = false;
  double rnorm = 0.0;
  double best_r = 1e300;
  int best_it = 0;
  for (it = 1; it <= max_iter; ++it) {
    // subspace eigenproblem on the device
    CK(cudaMemcpyAsync(G, Gh.data(), 32 * 32 * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_jacobi_eigh(G, k, 32, evals, evecs, s));
    // y = evecs[:, 0] (row-major k x k): gather column 0 into dots
    std::vector<double> ev(k), Y((size_t)k * k);
    CK(cudaMemcpyAsync(ev.data(), evals, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(Y.data(), evecs, (size_t)k * k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    theta = ev[0];
    std::vector<double> y0(k);
    for (int i = 0; i < k; ++i) y0[i] = Y[(size_t)i * k + 0];
    CK(cudaMemcpyAsync(dots, y0.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(scal, &theta, sizeof(double), cudaMemcpyHostToDevice, s));
    // x = V y, hx = AV y, r = hx - theta x
    CK(launch_combine(c->psi.p, c->V.p, dots, k, n, 0.0, s));
    CK(launch_combine(c->hx.p, c->AV.p, dots, k, n, 0.0, s));
    CK(launch_residual(c->r.p, c->hx.p, c->psi.p, scal, n, s));
    CK(launch_dots(c->r.p, 1, n, c->r.p, c->partial.p, scal + 1, s));
    double r2;
    CK(cudaMemcpyAsync(&r2, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rnorm = std::sqrt(std::max(r2, 0.0));
    if (rnorm <= std::max(tol, floor_rel * std::fabs(theta)) || k >= n) {
      conv = true;
      break;
    }
    // low-precision phase: once the residual is within reach of the low-precision
    // floor, stop when it no longer improves (further progress needs FP64 matvecs)
    if (floor_rel > 0.0) {
      if (rnorm < 0.5 * best_r) {
        best_r = rnorm;
        best_it = it;
      } else if (rnorm < 1e-5 * std::fabs(theta) && it - best_it >= 10) {
        conv = true;
        break;
      }
    }
    if (k == kmax) {
      // thick restart with the two lowest Ritz vectors
      const int keep = std::min(2, k);
      std::vector<double> yk((size_t)keep * k);
      for (int j = 0; j < keep; ++j)
        for (int i = 0; i < k; ++i) yk[(size_t)j * k + i] = Y[(size_t)i * k + j];
      DBuf<double> nv, nav, dy;
      nv.alloc((size_t)keep * n);
      nav.alloc((size_t)keep * n);
      dy.upload(yk, s);
      for (int j = 0; j < keep; ++j) {
        CK(launch_combine(nv.p + (int64_t)j * n, c->V.p, dy.p + (size_t)j * k, k, n, 0.0, s));
        CK(launch_combine(nav.p + (int64_t)j * n, c->AV.p, dy.p + (size_t)j * k, k, n, 0.0, s));
      }
      CK(cudaMemcpyAsync(c->V.p, nv.p, (size_t)keep * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(c->AV.p, nav.p, (size_t)keep * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      std::fill(Gh.begin(), Gh.end(), 0.0);
      for (int j = 0; j < keep; ++j) Gh[j * 32 + j] = ev[j];
      k = keep;
      CK(cudaStreamSynchronize(s));
    }
    // correction t = r / (theta - diag), orthogonalized against V twice
    CK(launch_precond(c->t.p, c->r.p, P.diag.p, scal, n, s));
    for (int pass = 0; pass < 2; ++pass) {
      CK(launch_dots(c->V.p, k, n, c->t.p, c->partial.p, dots, s));
      CK(launch_sub_proj(c->t.p, c->V.p, dots, k, n, s));
    }
    CK(launch_dots(c->t.p, 1, n, c->t.p, c->partial.p, scal + 1, s));
    double t2;
    CK(cudaMemcpyAsync(&t2, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(t2 > 1e-28)) {
      // preconditioned residual collapsed into the subspace: use the plain residual
      CK(cudaMemcpyAsync(c->t.p, c->r.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      for (int pass = 0; pass < 2; ++pass) {
        CK(launch_dots(c->V.p, k, n, c->t.p, c->partial.p, dots, s));
        CK(launch_sub_proj(c->t.p, c->V.p, dots, k, n, s));
      }
      CK(launch_dots(c->t.p, 1, n, c->t.p, c->partial.p, scal + 1, s));
      CK(cudaMemcpyAsync(&t2, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (!(t2 > 1e-28)) {
        conv = true;  // the subspace is invariant
        break;
      }
    }
    CK(launch_scale(c->t.p, scal + 1, 1, n, s));
    CK(cudaMemcpyAsync(c->V.p + (int64_t)k * n, c->t.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    hpsi_dev(c, c->V.p + (int64_t)k * n, c->AV.p + (int64_t)k * n, fp64);
    // new row/column of G: V^T (A v_k)
    CK(launch_dots(c->V.p, k + 1, n, c->AV.p + (int64_t)k * n, c->partial.p, dots, s));
    std::vector<double> col(k + 1);
    CK(cudaMemcpyAsync(col.data(), dots, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i <= k; ++i) {
      Gh[i * 32 + k] = col[i];
      Gh[k * 32 + i] = col[i];
    }
    ++k;
  }
  // normalize the Ritz vector once more
  normalize(c->psi.p);
  c->last_resid = rnorm;
  CK(cudaStreamSynchronize(s));
  c->psi_valid = true;
  c->dav_iters += std::min(it, max_iter);
  if (energy) *energy = theta;
  if (iters) *iters = std::min(it, max_iter);
}

// Refinement of a low-precision Ritz vector x to an FP64 residual (defect
// correction inside Davidson).  Each outer step applies H to x in FP64 (the
// exact residual r = Hx - theta x, the convergence test and the Rayleigh
// quotient theta), then expands the subspace [x, t_1, t_2, ...] with
// low-precision matvecs only.  The coupling of x to the corrections is taken
// from the exact Hx (G_0i = (Hx) . t_i, by symmetry), so the low-precision
// error enters only through the t_i^T H t_j block, i.e. scaled by the size of
// the correction: each outer step reduces the residual by about the
// low-precision accuracy times ||H|| / gap instead of stalling at it.
// Returns false if the exact residual stopped improving (the caller then
// finishes with FP64 matvecs).
static bool davidson_refine(dmrg_ctx *c, double tol, int max_iter, double *energy, int *iters,
                            int *iters_lowp, bool &conv) {
  build_hplan(c);
  HPlan &P = c->plan;
  const int64_t n = P.psi.dim;
  const int kmax = (int)std::min<int64_t>(24, std::max<int64_t>(n, 1));
  c->V.alloc((size_t)kmax * n);
  c->AV.alloc((size_t)kmax * n);
  c->r.alloc(n);
  c->t.alloc(n);
  c->hx.alloc(n);
  c->partial.alloc((size_t)dots_partial_blocks(n) * 32);
  c->small.alloc(4096);
  double *G = c->small.p, *evals = c->small.p + 1024, *evecs = c->small.p + 1056;
  double *dots = c->small.p + 2200, *scal = c->small.p + 2300, *dot0 = c->small.p + 2400;
  cudaStream_t s = c->stream;
  auto get = [&](const double *d) {
    double v;
    CK(cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return v;
  };
  auto norm2 = [&](const double *x) {
    CK(launch_dots(x, 1, n, x, c->partial.p, scal + 1, s));
    return get(scal + 1);
  };
  CK(cudaMemcpyAsync(c->V.p, c->psi.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(launch_dots(c->V.p, 1, n, c->V.p, c->partial.p, scal + 1, s));
  CK(launch_scale(c->V.p, scal + 1, 1, n, s));
  int it = 0, itl = 0, stalls = 0;
  double theta = 0.0, best = 1e300;
  bool ok = true;
  conv = false;
  std::vector<double> Gh(32 * 32, 0.0);
  // thick restart (refine_keep > 0): the next Ritz vectors of an outer step's
  // subspace and their low-precision images join x in the next outer step
  const int keep = std::min(c->refine_keep, kmax - 2);
  DBuf<double> Xv, Xa;
  int nx = 0;
  if (keep > 0) {
    Xv.alloc((size_t)keep * n);
    Xa.alloc((size_t)keep * n);
  }
  std::vector<double> Ylast;
  int klast = 0;
  for (;;) {
    // ---- outer step: exact H x, theta, residual
    hpsi_dev(c, c->V.p, c->AV.p, true);
    ++it;
    CK(launch_dots(c->V.p, 1, n, c->AV.p, c->partial.p, dots, s));
    theta = get(dots);
    CK(cudaMemcpyAsync(scal, &theta, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_residual(c->r.p, c->AV.p, c->V.p, scal, n, s));
    const double rnorm = std::sqrt(std::max(norm2(c->r.p), 0.0));
    c->last_resid = rnorm;
    if (rnorm <= tol) {
      conv = true;
      break;
    }
    if (rnorm < 0.5 * best) {
      best = rnorm;
      stalls = 0;
    } else if (++stalls >= 2) {
      ok = false;
      break;
    }
    if (it >= max_iter) break;
    std::fill(Gh.begin(), Gh.end(), 0.0);
    Gh[0] = theta;
    int k = 1;
    bool solved = false;
    for (int j = 0; j < nx && k < kmax - 1; ++j) {
      double *vk = c->V.p + (int64_t)k * n, *ak = c->AV.p + (int64_t)k * n;
      CK(cudaMemcpyAsync(vk, Xv.p + (int64_t)j * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ak, Xa.p + (int64_t)j * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      for (int pass = 0; pass < 2; ++pass) {  // orthogonal to V[0..k); the image follows
        CK(launch_dots(c->V.p, k, n, vk, c->partial.p, dots, s));
        CK(launch_sub_proj(vk, c->V.p, dots, k, n, s));
        CK(launch_sub_proj(ak, c->AV.p, dots, k, n, s));
      }
      if (!(norm2(vk) > 1e-16)) continue;  // leaves |vk|^2 in scal[1]
      CK(launch_scale(vk, scal + 1, 1, n, s));
      CK(launch_scale(ak, scal + 1, 1, n, s));
      CK(launch_dots(c->V.p, k + 1, n, ak, c->partial.p, dots, s));
      CK(launch_dots(c->AV.p, 1, n, vk, c->partial.p, dot0, s));  // exact (H x) . v
      std::vector<double> col(k + 1);
      CK(cudaMemcpyAsync(col.data(), dots, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(col.data(), dot0, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int i = 0; i <= k; ++i) {
        Gh[i * 32 + k] = col[i];
        Gh[k * 32 + i] = col[i];
      }
      ++k;
    }
    // ---- inner expansion with low-precision matvecs
    for (;;) {
      CK(launch_precond(c->t.p, c->r.p, P.diag.p, scal, n, s));
      double t2 = 0.0;
      for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) CK(cudaMemcpyAsync(c->t.p, c->r.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int pass = 0; pass < 2; ++pass) {
          CK(launch_dots(c->V.p, k, n, c->t.p, c->partial.p, dots, s));
          CK(launch_sub_proj(c->t.p, c->V.p, dots, k, n, s));
        }
        t2 = norm2(c->t.p);
        if (t2 > 1e-28) break;
      }
      if (!(t2 > 1e-28)) break;  // nothing new to add: take the current Ritz vector
      CK(launch_scale(c->t.p, scal + 1, 1, n, s));
      CK(cudaMemcpyAsync(c->V.p + (int64_t)k * n, c->t.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      hpsi_dev(c, c->V.p + (int64_t)k * n, c->AV.p + (int64_t)k * n, false);
      ++it;
      ++itl;
      CK(launch_dots(c->V.p, k + 1, n, c->AV.p + (int64_t)k * n, c->partial.p, dots, s));
      CK(launch_dots(c->AV.p, 1, n, c->t.p, c->partial.p, dot0, s));  // exact (H x) . t
      std::vector<double> col(k + 1);
      CK(cudaMemcpyAsync(col.data(), dots, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(col.data(), dot0, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int i = 0; i <= k; ++i) {
        Gh[i * 32 + k] = col[i];
        Gh[k * 32 + i] = col[i];
      }
      ++k;
      // Ritz pair of the subspace; estimated residual
      CK(cudaMemcpyAsync(G, Gh.data(), 32 * 32 * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(launch_jacobi_eigh(G, k, 32, evals, evecs, s));
      std::vector<double> Y((size_t)k * k);
      double th;
      CK(cudaMemcpyAsync(&th, evals, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(Y.data(), evecs, (size_t)k * k * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      solved = true;
      if (keep > 0) {
        Ylast = Y;
        klast = k;
      }
      std::vector<double> y0(k);
      for (int i = 0; i < k; ++i) y0[i] = Y[(size_t)i * k];
      CK(cudaMemcpyAsync(dots, y0.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(scal, &th, sizeof(double), cudaMemcpyHostToDevice, s));
      CK(launch_combine(c->psi.p, c->V.p, dots, k, n, 0.0, s));
      CK(launch_combine(c->hx.p, c->AV.p, dots, k, n, 0.0, s));
      CK(launch_residual(c->r.p, c->hx.p, c->psi.p, scal, n, s));
      const double rest = std::sqrt(std::max(norm2(c->r.p), 0.0));
      if (rest <= std::max(0.01 * rnorm, 0.5 * tol) || k == kmax || it >= max_iter) break;
    }
    if (k == 1 || (keep > 0 && !solved)) {
      ok = false;  // the subspace could not grow
      break;
    }
    if (keep > 0) {  // next Ritz vectors of this subspace and their images, for the next step
      nx = std::min(keep, klast - 1);
      for (int j = 0; j < nx; ++j) {
        std::vector<double> yj(klast);
        for (int i = 0; i < klast; ++i) yj[i] = Ylast[(size_t)i * klast + (j + 1)];
        CK(cudaMemcpyAsync(dots, yj.data(), klast * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(launch_combine(Xv.p + (int64_t)j * n, c->V.p, dots, klast, n, 0.0, s));
        CK(launch_combine(Xa.p + (int64_t)j * n, c->AV.p, dots, klast, n, 0.0, s));
        CK(cudaStreamSynchronize(s));  // yj is released at the end of the iteration
      }
    }
    // the Ritz vector becomes x of the next outer step
    CK(cudaMemcpyAsync(c->V.p, c->psi.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(launch_dots(c->V.p, 1, n, c->V.p, c->partial.p, scal + 1, s));
    CK(launch_scale(c->V.p, scal + 1, 1, n, s));
  }
  CK(cudaMemcpyAsync(c->psi.p, c->V.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  c->psi_valid = true;
  c->dav_iters += it;
  if (energy) *energy = theta;
  if (iters) *iters = it;
  if (iters_lowp) *iters_lowp = itl;
  return ok;
}

// Davidson at the working precision.  In mixed precision the low-precision
// matvecs run down to their attainable residual (~1e-6 |E|), then the
// defect-corrected refinement above reaches the requested tolerance with a
// few FP64 matvecs (plain FP64 Davidson finishes if it stalls), so the
// energy and vector are FP64 quality.
static void davidson(dmrg_ctx *c, double tol, int max_iter, double *energy, int *iters, bool &conv) {
  build_hplan(c);
  if (!c->plan.lowp) {
    davidson_core(c, tol, 0.0, max_iter, true, energy, iters, conv);
    return;
  }
  int it1 = 0, it2 = 0, it2l = 0, it3 = 0;
  double e = 0.0;
  // the low-precision phase hands over well above its attainable residual
  // (~1e-7 |E| for FP32, ~1e-5 |E| for split-BF16): the refinement below
  // converges from there with a few FP64 matvecs, while iterating into the
  // floor only burns low-precision matvecs
  const double handover = c->prec == DMRG_PREC_BF16X3 ? 1e-4 : 1e-6;
  davidson_core(c, tol, handover, max_iter, false, &e, &it1, conv);
  c->dav_iters_lowp += it1;
  const bool ok = davidson_refine(c, tol, std::max(1, max_iter - it1), &e, &it2, &it2l, conv);
  c->dav_iters_lowp += it2l;
  if (!ok && !conv && it1 + it2 < max_iter)
    davidson_core(c, tol, 0.0, max_iter - it1 - it2, true, &e, &it3, conv);
  if (energy) *energy = e;
  if (iters) *iters = it1 + it2 + it3;
}

}  // namespace dmrg

using namespace dmrg;

#define API_BEGIN try {
#define API_END                                                  \
  }                                                              \
  catch (const Fail &f) {                                        \
    set_error(f.msg);                                            \
    return f.code;                                               \
  }                                                              \
  catch (const std::bad_alloc &) {                               \
    set_error("host allocation failed");                         \
    return DMRG_ENOMEM;                                          \
  }                                                              \
  catch (const std::exception &e) {                              \
    set_error(e.what());                                         \
    return DMRG_EINVAL;                                          \
  }                                                              \
  return DMRG_OK;

extern "C" int dmrg_init(int L, int N, int two_sz, const double *h, const double *v, int M,
                         int precision, void *cuda_stream, dmrg_ctx **out) {
  API_BEGIN
  if (!out) throw Fail{DMRG_EINVAL, "out is NULL"};
  *out = nullptr;
  if (L < 2) throw Fail{DMRG_EINVAL, "L must be >= 2"};
  if (N < 0 || N > 2 * L) throw Fail{DMRG_EINVAL, "N out of range"};
  if (std::abs(two_sz) > N || ((N - two_sz) & 1)) throw Fail{DMRG_EINVAL, "two_sz incompatible with N"};
  const int nu = (N + two_sz) / 2, nd = (N - two_sz) / 2;
  if (nu > L || nd > L) throw Fail{DMRG_EINVAL, "more electrons of one spin than orbitals"};
  if (M < 1) throw Fail{DMRG_EINVAL, "M must be >= 1"};
  if (precision != DMRG_PREC_FP64 && precision != DMRG_PREC_FP32 && precision != DMRG_PREC_BF16X3)
    throw Fail{DMRG_EINVAL, "unknown precision"};
  if (!h || !v) throw Fail{DMRG_EINVAL, "integrals are NULL"};
  const size_t L2 = (size_t)L * L, L4 = L2 * L2;
  for (size_t i = 0; i < L2; ++i)
    if (!std::isfinite(h[i])) throw Fail{DMRG_EINVAL, "h has a non-finite entry"};
  for (size_t i = 0; i < L4; ++i)
    if (!std::isfinite(v[i])) throw Fail{DMRG_EINVAL, "v has a non-finite entry"};
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      if (std::fabs(h[i * L + j] - h[j * L + i]) > 1e-12) throw Fail{DMRG_EINVAL, "h is not symmetric"};
  auto c = std::make_unique<dmrg_ctx>();
  c->L = L;
  c->N = N;
  c->nu = nu;
  c->nd = nd;
  c->M = M;
  c->M_bwd = M;
  c->prec = precision;
  c->stream = (cudaStream_t)cuda_stream;
  c->I.L = L;
  c->I.h.assign(h, h + L2);
  c->I.v.assign(v, v + L4);
  c->dstatus.alloc(8);  // flag + time-out record of the tensor-core kernel
  CK(cudaMemsetAsync(c->dstatus.p, 0, 8 * sizeof(int), c->stream));
  c->left.resize(L);
  c->right.resize(L);
  c->left[0] = empty_block(0, L);
  c->right[0] = empty_block(1, L);
  // Aufbau product state: right blocks right-to-left with one kept state each
  for (int k = L - 2; k >= 1; --k) {
    c->k = k;
    DevBlock *r = rblock(c.get());
    Enlarged enl = enlarged(r->lay, -1);
    const int s = k + 1;
    const int st = (s < nu ? 1 : 0) + (s < nd ? 2 : 0);
    std::vector<int> kept(enl.size(), 0);
    std::vector<double> O;
    for (size_t e = 0; e < enl.size(); ++e)
      for (auto &sb : enl[e].sub)
        if (sb.x == st) {
          kept[e] = 1;
          O.assign((size_t)enl[e].dim, 0.0);
          O[sb.roff] = 1.0;
        }
    // a single kept sector: O is its column
    // (dmrg_renormalize expects all sectors concatenated; others keep 0 columns)
    DBuf<double> Odev;
    std::vector<int64_t> Ooff(enl.size(), 0);
    Odev.upload(O, c->stream);
    auto nb = renormalize_block(c.get(), -1, enl, kept, Odev, Ooff);
    c->right[L - k - 1] = std::move(nb);
  }
  c->k = 0;
  c->dir = 1;
  c->launch_base = kernel_launch_count();
  *out = c.release();
  API_END
}

extern "C" int dmrg_free(dmrg_ctx *c) {
  if (!c) return DMRG_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->solver) cusolverDnDestroy(c->solver);
  for (auto e : c->ev) cudaEventDestroy(e);
  delete c;
  return DMRG_OK;
}

extern "C" int dmrg_set_bond_dims(dmrg_ctx *c, int m_forward, int m_backward) {
  API_BEGIN
  if (!c || m_forward < 1 || m_backward < 1) throw Fail{DMRG_EINVAL, "dmrg_set_bond_dims: NULL or M < 1"};
  c->M = m_forward;
  c->M_bwd = m_backward;
  API_END
}

extern "C" int dmrg_set_precision(dmrg_ctx *c, int precision) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "context is NULL"};
  if (precision != DMRG_PREC_FP64 && precision != DMRG_PREC_FP32 && precision != DMRG_PREC_BF16X3)
    throw Fail{DMRG_EINVAL, "unknown precision"};
  if (precision != c->prec) {
    CK(cudaStreamSynchronize(c->stream));
    c->prec = precision;
    c->plan.valid = false;  // task lists and low-precision copies are rebuilt on next use
    c->plan.chain32.release();  // the old working precision's copies, tiles and task list
    for (auto &f : c->plan.f32) f.release();
    ++c->plan_gen;
  }
  API_END
}

extern "C" int dmrg_release_block(dmrg_ctx *c, int side, int sites) {
  API_BEGIN
  if (!c || (side != 0 && side != 1) || sites < 1 || sites > c->L - 2)
    throw Fail{DMRG_EINVAL, "dmrg_release_block: side 0 or 1, 1 <= sites <= L-2"};
  const int used = side == 0 ? c->k : c->L - c->k - 2;
  if (sites == used) throw Fail{DMRG_EINVAL, "dmrg_release_block: the block is used at the current position"};
  auto &store = side == 0 ? c->left : c->right;
  if (sites < (int)store.size() && store[sites]) {
    CK(cudaStreamSynchronize(c->stream));  // no launch in flight still reads it
    store[sites].reset();
  }
  API_END
}

extern "C" int dmrg_set_position(dmrg_ctx *c, int k, int direction) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "ctx is NULL"};
  if (k < 0 || k > c->L - 2) throw Fail{DMRG_EINVAL, "position out of range"};
  if (direction != 1 && direction != -1) throw Fail{DMRG_EINVAL, "direction must be +1 or -1"};
  if (k != c->k) {
    c->plan.valid = false;
    c->psi_valid = false;
  }
  c->k = k;
  c->dir = direction;
  API_END
}

extern "C" int dmrg_get_position(dmrg_ctx *c, int *k, int *direction) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "ctx is NULL"};
  if (k) *k = c->k;
  if (direction) *direction = c->dir;
  API_END
}

extern "C" int dmrg_psi_layout(dmrg_ctx *c, int *nblocks, int *blocks, long long *dim) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "ctx is NULL"};
  require_blocks(c);
  Psi P = psi_layout(lblock(c)->lay, rblock(c)->lay, c->nu, c->nd);
  if (nblocks) *nblocks = (int)P.blk.size();
  if (dim) *dim = P.dim;
  if (blocks)
    for (size_t i = 0; i < P.blk.size(); ++i) {
      const PsiBlock &b = P.blk[i];
      int *o = blocks + 7 * i;
      o[0] = b.a; o[1] = b.b; o[2] = b.c; o[3] = b.d; o[4] = b.ma; o[5] = b.md; o[6] = (int)b.off;
    }
  API_END
}

extern "C" int dmrg_block_sectors(dmrg_ctx *c, int side, int *nsec, int *sectors) {
  API_BEGIN
  if (!c || (side != 0 && side != 1)) throw Fail{DMRG_EINVAL, "bad arguments"};
  DevBlock *b = side == 0 ? lblock(c) : rblock(c);
  if (!b) throw Fail{DMRG_ESTATE, "block not built"};
  if (nsec) *nsec = (int)b->lay.sec.size();
  if (sectors)
    for (size_t i = 0; i < b->lay.sec.size(); ++i) {
      sectors[3 * i] = b->lay.sec[i].nu;
      sectors[3 * i + 1] = b->lay.sec[i].nd;
      sectors[3 * i + 2] = b->lay.sec[i].dim;
    }
  API_END
}

extern "C" int dmrg_enlarged_layout(dmrg_ctx *c, int direction, int *nsec, int *sectors) {
  API_BEGIN
  if (!c || (direction != 1 && direction != -1)) throw Fail{DMRG_EINVAL, "bad arguments"};
  DevBlock *b = direction > 0 ? lblock(c) : rblock(c);
  if (!b) throw Fail{DMRG_ESTATE, "block not built"};
  Enlarged e = enlarged(b->lay, direction);
  if (nsec) *nsec = (int)e.size();
  if (sectors)
    for (size_t i = 0; i < e.size(); ++i) {
      sectors[3 * i] = e[i].nu;
      sectors[3 * i + 1] = e[i].nd;
      sectors[3 * i + 2] = e[i].dim;
    }
  API_END
}

extern "C" int dmrg_hpsi(dmrg_ctx *c, const double *psi, double *sigma, int device_ptrs) {
  API_BEGIN
  if (!c || !psi || !sigma) throw Fail{DMRG_EINVAL, "NULL argument"};
  build_hplan(c);
  const int64_t n = c->plan.psi.dim;
  if (device_ptrs) {
    hpsi_dev(c, psi, sigma);
  } else {
    DBuf<double> dp, ds;
    dp.alloc(n);
    ds.alloc(n);
    CK(cudaMemcpyAsync(dp.p, psi, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    hpsi_dev(c, dp.p, ds.p);
    CK(cudaMemcpyAsync(sigma, ds.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  check_status(c);
  API_END
}

extern "C" int dmrg_hpsi_flops(dmrg_ctx *c, double *flops, long long *tasks) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "ctx is NULL"};
  build_hplan(c);
  if (flops) *flops = c->plan.flops;
  if (tasks) *tasks = c->plan.ntasks;
  API_END
}

extern "C" int dmrg_set_psi(dmrg_ctx *c, const double *psi, int device_ptr) {
  API_BEGIN
  if (!c || !psi) throw Fail{DMRG_EINVAL, "NULL argument"};
  build_hplan(c);
  const int64_t n = c->plan.psi.dim;
  c->psi.alloc(n);
  CK(cudaMemcpyAsync(c->psi.p, psi, n * sizeof(double),
                     device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  if (!device_ptr) CK(cudaStreamSynchronize(c->stream));
  c->psi_valid = true;
  API_END
}

extern "C" int dmrg_get_psi(dmrg_ctx *c, double *psi, int device_ptr) {
  API_BEGIN
  if (!c || !psi) throw Fail{DMRG_EINVAL, "NULL argument"};
  if (!c->psi_valid) throw Fail{DMRG_ESTATE, "no wave function at this position"};
  build_hplan(c);
  CK(cudaMemcpyAsync(psi, c->psi.p, c->plan.psi.dim * sizeof(double),
                     device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!device_ptr) CK(cudaStreamSynchronize(c->stream));
  API_END
}

extern "C" int dmrg_davidson(dmrg_ctx *c, double tol, int max_iter, double *energy, int *iters) {
  API_BEGIN
  if (!c || !(tol > 0.0) || max_iter < 1) throw Fail{DMRG_EINVAL, "bad arguments"};
  bool conv = false;
  davidson(c, tol, max_iter, energy, iters, conv);
  check_status(c);
  if (!conv) throw Fail{DMRG_ENOCONV, "Davidson did not reach the tolerance"};
  API_END
}

extern "C" int dmrg_davidson_lowp(dmrg_ctx *c, double tol, int max_iter, double *energy, int *iters) {
  API_BEGIN
  if (!c || !(tol > 0.0) || max_iter < 1) throw Fail{DMRG_EINVAL, "bad arguments"};
  build_hplan(c);
  bool conv = false;
  const long long h0 = c->hpsi_calls;
  davidson_core(c, tol, 0.0, max_iter, !c->plan.lowp, energy, nullptr, conv);
  if (c->plan.lowp) c->dav_iters_lowp += c->hpsi_calls - h0;
  if (iters) *iters = (int)(c->hpsi_calls - h0);
  check_status(c);
  if (!conv) throw Fail{DMRG_ENOCONV, "Davidson did not reach the tolerance"};
  API_END
}

extern "C" int dmrg_renormalize(dmrg_ctx *c, int direction, const int *kept, const double *O,
                                double *discarded_weight) {
  API_BEGIN
  if (!c || (direction != 1 && direction != -1)) throw Fail{DMRG_EINVAL, "bad arguments"};
  do_renormalize(c, direction, O ? kept : nullptr, O, discarded_weight, O ? nullptr : const_cast<int *>(kept));
  API_END
}

// The two-site entropies of the current wave function (host copy of psi).
static void current_entropies(dmrg_ctx *c, double s3[3], double *rho2);

// Sweeps (Sec. 2.1): forward over positions 0..L-3, backward over L-2..1, a
// Davidson step then a truncation + renormalization at each.  Per step j
// (optional records): energies[j], the discarded weight of its truncation,
// and the entropies of the step's two sites {s_k, s_k+1, s_pair}.
static void sweep_impl(dmrg_ctx *c, int nsweeps, double tol, double *energies, double *discarded,
                       double *entropies) {
  c->k = 0;
  c->dir = 1;
  c->plan.valid = false;
  int idx = 0;
  auto step = [&](int direction) {
    double e, dw = 0.0;
    int it;
    bool conv;
    davidson(c, tol, c->sweep_max_iter, &e, &it, conv);
    if (energies) energies[idx] = e;
    if (entropies) current_entropies(c, entropies + 3 * idx, nullptr);
    do_renormalize(c, direction, nullptr, nullptr, &dw, nullptr);
    if (discarded) discarded[idx] = dw;
    ++idx;
  };
  for (int sw = 0; sw < nsweeps; ++sw) {
    for (int k = 0; k <= c->L - 3; ++k) step(+1);
    for (int k = c->L - 2; k >= 1; --k) step(-1);
  }
}

extern "C" int dmrg_sweep(dmrg_ctx *c, int nsweeps, double tol, double *energies) {
  API_BEGIN
  if (!c || nsweeps < 0 || !(tol > 0.0)) throw Fail{DMRG_EINVAL, "bad arguments"};
  if (c->L < 3) throw Fail{DMRG_EINVAL, "sweeps need L >= 3"};
  sweep_impl(c, nsweeps, tol, energies, nullptr, nullptr);
  API_END
}

extern "C" int dmrg_sweep_record(dmrg_ctx *c, int nsweeps, double tol, double *energies, double *discarded,
                                 double *entropies) {
  API_BEGIN
  if (!c || nsweeps < 0 || !(tol > 0.0)) throw Fail{DMRG_EINVAL, "bad arguments"};
  if (c->L < 3) throw Fail{DMRG_EINVAL, "sweeps need L >= 3"};
  sweep_impl(c, nsweeps, tol, energies, discarded, entropies);
  API_END
}

extern "C" int dmrg_block_op(dmrg_ctx *c, int side, int kind, int i, int j, double *out,
                             long long *n) {
  API_BEGIN
  if (!c || (side != 0 && side != 1)) throw Fail{DMRG_EINVAL, "bad arguments"};
  DevBlock *b = side == 0 ? lblock(c) : rblock(c);
  if (!b) throw Fail{DMRG_ESTATE, "block not built"};
  int f, kk;
  if (!b->lay.get(kind, i, j, f, kk)) throw Fail{DMRG_EINVAL, "no such stored operator"};
  const Family &F = b->lay.fam[f];
  int64_t tot = 0;
  for (int a = 0; a < (int)b->lay.sec.size(); ++a)
    if (F.bra[a] >= 0) tot += (int64_t)b->lay.sec[F.bra[a]].dim * b->lay.sec[a].dim;
  if (n) *n = tot;
  if (out) {
    int64_t pos = 0;
    for (int a = 0; a < (int)b->lay.sec.size(); ++a) {
      if (F.bra[a] < 0) continue;
      const int64_t sz = (int64_t)b->lay.sec[F.bra[a]].dim * b->lay.sec[a].dim;
      CK(cudaMemcpyAsync(out + pos, b->ops.p + F.base + F.off[a] + kk * sz, sz * sizeof(double),
                         cudaMemcpyDeviceToHost, c->stream));
      pos += sz;
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  API_END
}

extern "C" int dmrg_stats(dmrg_ctx *c, int reset, double *hpsi_ms, long long *hpsi_calls,
                          double *hpsi_flops, long long *kernel_launches, long long *davidson_iters,
                          long long *davidson_iters_lowp, double *last_residual) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "ctx is NULL"};
  fold_events(c);
  if (hpsi_ms) *hpsi_ms = c->hpsi_ms_folded;
  if (hpsi_calls) *hpsi_calls = c->hpsi_calls;
  if (hpsi_flops) *hpsi_flops = c->hpsi_flops_acc;
  if (kernel_launches) *kernel_launches = kernel_launch_count() - c->launch_base;
  if (davidson_iters) *davidson_iters = c->dav_iters;
  if (davidson_iters_lowp) *davidson_iters_lowp = c->dav_iters_lowp;
  if (last_residual) *last_residual = c->last_resid;
  if (reset) {
    c->dav_iters_lowp = 0;
    c->hpsi_ms_folded = 0.0;
    c->hpsi_calls = 0;
    c->hpsi_flops_acc = 0.0;
    c->dav_iters = 0;
    c->launch_base = kernel_launch_count();
  }
  API_END
}

extern "C" int dmrg_plan_hpsi_flops(int L, int N, int two_sz, const double *h, const double *v, int k,
                                    int nl, const int *sec_l, int nr, const int *sec_r, double *flops,
                                    long long *tasks) {
  API_BEGIN
  if (L < 2 || k < 0 || k > L - 2 || !h || !v || nl < 1 || nr < 1 || !sec_l || !sec_r)
    throw Fail{DMRG_EINVAL, "dmrg_plan_hpsi_flops: bad arguments"};
  if (std::abs(two_sz) > N || ((N - two_sz) & 1)) throw Fail{DMRG_EINVAL, "two_sz incompatible with N"};
  Integrals I;
  I.L = L;
  I.h.assign(h, h + (size_t)L * L);
  I.v.assign(v, v + (size_t)L * L * L * L);
  auto sectors = [](int n, const int *t) {
    std::vector<Sector> out;
    for (int i = 0; i < n; ++i) out.push_back({t[3 * i], t[3 * i + 1], t[3 * i + 2]});
    return out;
  };
  std::vector<int> ls, rs;
  for (int s = 0; s < k; ++s) ls.push_back(s);
  for (int s = k + 2; s < L; ++s) rs.push_back(s);
  BlockLayout lb, rb;
  build_layout(lb, 0, L, ls, sectors(nl, sec_l));
  build_layout(rb, 1, L, rs, sectors(nr, sec_r));
  Psi Y = psi_layout(lb, rb, (N + two_sz) / 2, (N - two_sz) / 2);
  TempSet temps;
  auto rps = resolve_pieces(I, k, lb, rb, temps);
  const BlockLayout *lay[2] = {&lb, &rb};
  temps.layout(lay);
  Arenas A{{&lb, &rb}, {nullptr, nullptr}, &temps, {nullptr, nullptr}, 8};
  ChainList CL;
  double f = 0.0;
  expand_hpsi_grouped(rps, A, Y, lb, CL, f);
  if (flops) *flops = f;
  if (tasks) *tasks = (long long)CL.flat.size();
  API_END
}

extern "C" int dmrg_debug_tasks(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                                const int *sec_l, int nr, const int *sec_r, int grouped, int *out,
                                long long cap, long long *ntasks) {
  API_BEGIN
  if (L < 2 || k < 0 || k > L - 2 || !h || !v || nl < 1 || nr < 1 || !sec_l || !sec_r || !ntasks)
    throw Fail{DMRG_EINVAL, "dmrg_debug_tasks: bad arguments"};
  if (std::abs(two_sz) > N || ((N - two_sz) & 1)) throw Fail{DMRG_EINVAL, "two_sz incompatible with N"};
  Integrals I;
  I.L = L;
  I.h.assign(h, h + (size_t)L * L);
  I.v.assign(v, v + (size_t)L * L * L * L);
  auto sectors = [](int n, const int *t) {
    std::vector<Sector> o;
    for (int i = 0; i < n; ++i) o.push_back({t[3 * i], t[3 * i + 1], t[3 * i + 2]});
    return o;
  };
  std::vector<int> ls, rs;
  for (int s = 0; s < k; ++s) ls.push_back(s);
  for (int s = k + 2; s < L; ++s) rs.push_back(s);
  BlockLayout lb, rb;
  build_layout(lb, 0, L, ls, sectors(nl, sec_l));
  build_layout(rb, 1, L, rs, sectors(nr, sec_r));
  Psi Y = psi_layout(lb, rb, (N + two_sz) / 2, (N - two_sz) / 2);
  TempSet temps;
  auto rps = resolve_pieces(I, k, lb, rb, temps);
  const BlockLayout *lay[2] = {&lb, &rb};
  temps.layout(lay);
  Arenas A{{&lb, &rb}, {nullptr, nullptr}, &temps, {nullptr, nullptr}, 8};
  ChainList CL;
  double f = 0.0;
  ChainList::Keyed tasks;
  if (grouped) {  // the task list the GPU runs: grouped by output block
    expand_hpsi_grouped(rps, A, Y, lb, CL, f);
    *ntasks = (long long)CL.flat.size();
    for (const auto &g : CL.grp)
      for (int i = g.first; i < g.first + g.count; ++i) tasks.push_back({Y.find_block(g.d), CL.flat[i]});
  } else {  // build order
    expand_hpsi(rps, A, Y, lb, CL, f);
    *ntasks = (long long)CL.size();
    for (const auto &p : CL.parts) tasks.insert(tasks.end(), p.begin(), p.end());
  }
  if (out) {
    if (cap < *ntasks) throw Fail{DMRG_EINVAL, "dmrg_debug_tasks: buffer too small"};
    for (size_t i = 0; i < tasks.size(); ++i) {
      const int g = tasks[i].first;
      const ChainEntry &e = tasks[i].second;
      int *o = out + 7 * i;
      o[0] = g;
      o[1] = Y.blk[g].ma;  // m
      o[2] = e.n;
      o[3] = e.p;
      o[4] = Y.blk[g].md;  // q
      o[5] = (e.x == ~0ull ? 1 : 0) | (e.z == ~0ull ? 2 : 0);
      o[6] = (int)e.y;     // input block offset in psi
    }
  }
  API_END
}

extern "C" int dmrg_debug_exec(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                               const int *sec_l, int nr, const int *sec_r, int tensor_cores,
                               const double *tune, long long *counts, long long *xs_out, long long *grp_out,
                               long long *red_out) {
  API_BEGIN
  if (L < 2 || k < 0 || k > L - 2 || !h || !v || nl < 1 || nr < 1 || !sec_l || !sec_r || !counts)
    throw Fail{DMRG_EINVAL, "dmrg_debug_exec: bad arguments"};
  if (std::abs(two_sz) > N || ((N - two_sz) & 1)) throw Fail{DMRG_EINVAL, "two_sz incompatible with N"};
  ChainTune T;
  if (tune) {
    if (!(tune[0] >= 1.0) || !(tune[1] >= 0.0) || tune[2] < 1 || tune[2] > 129 || (tune[3] != 0 && tune[3] != 1) ||
        (tune[4] != 0 && tune[4] != 1))
      throw Fail{DMRG_EINVAL, "dmrg_debug_exec: bad launch-shape parameters"};
    T.target_chunks = tune[0];
    T.min_chunk = tune[1];
    T.tc_min = (int)tune[2];
    T.by_work = (int)tune[3];
    T.tc_tiny = (int)tune[4];
  }
  Integrals I;
  I.L = L;
  I.h.assign(h, h + (size_t)L * L);
  I.v.assign(v, v + (size_t)L * L * L * L);
  auto sectors = [](int n, const int *t) {
    std::vector<Sector> out;
    for (int i = 0; i < n; ++i) out.push_back({t[3 * i], t[3 * i + 1], t[3 * i + 2]});
    return out;
  };
  std::vector<int> ls, rs;
  for (int s = 0; s < k; ++s) ls.push_back(s);
  for (int s = k + 2; s < L; ++s) rs.push_back(s);
  BlockLayout lb, rb;
  build_layout(lb, 0, L, ls, sectors(nl, sec_l));
  build_layout(rb, 1, L, rs, sectors(nr, sec_r));
  Psi Y = psi_layout(lb, rb, (N + two_sz) / 2, (N - two_sz) / 2);
  TempSet temps;
  auto rps = resolve_pieces(I, k, lb, rb, temps);
  const BlockLayout *lay[2] = {&lb, &rb};
  temps.layout(lay);
  Arenas A{{&lb, &rb}, {nullptr, nullptr}, &temps, {nullptr, nullptr}, 8};
  ChainList CL;
  double f = 0.0;
  expand_hpsi_grouped(rps, A, Y, lb, CL, f);
  ExecPlan X;
  plan_exec(CL, tensor_cores != 0, true, T, X);
  counts[0] = (long long)X.xs.size();
  counts[1] = (long long)X.vb.size();
  counts[2] = (long long)X.vf.size();
  counts[3] = (long long)X.vt.size();
  counts[4] = (long long)X.vr.size();
  counts[5] = X.tiles;
  counts[6] = X.soff;
  counts[7] = X.e0;
  if (xs_out)
    for (size_t i = 0; i < X.xs.size(); ++i) {
      const ChainEntry &e = X.xs[i];
      long long *o = xs_out + 8 * i;
      o[0] = (long long)e.y;
      o[1] = e.n;
      o[2] = e.p;
      o[3] = e.yrs;
      o[4] = e.ycs;
      o[5] = (e.x == ~0ull ? 1 : 0) | (e.z == ~0ull ? 2 : 0);
      o[6] = (long long)e.x;  // -1: identity
      o[7] = (long long)e.z;
    }
  if (grp_out) {
    size_t j = 0;
    const std::vector<ChainGroup> *kinds[3] = {&X.vb, &X.vf, &X.vt};
    for (int kd = 0; kd < 3; ++kd)
      for (const ChainGroup &g : *kinds[kd]) {
        long long *o = grp_out + 8 * j++;
        o[0] = kd;
        o[1] = (long long)g.d;
        o[2] = g.drs;
        o[3] = g.dcs;
        o[4] = g.m;
        o[5] = g.q;
        o[6] = g.first;
        o[7] = g.count;
      }
  }
  if (red_out)
    for (size_t i = 0; i < X.vr.size(); ++i) {
      const ReduceGroup &r = X.vr[i];
      long long *o = red_out + 8 * i;
      o[0] = r.e0;
      o[1] = r.soff;
      o[2] = (long long)r.d;
      o[3] = r.drs;
      o[4] = r.dcs;
      o[5] = r.m;
      o[6] = r.q;
      o[7] = r.nsplit;
    }
  API_END
}

extern "C" int dmrg_debug_validate(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                                   const int *sec_l, int nr, const int *sec_r, int tensor_cores,
                                   const double *tune, long long *checked, long long *bad) {
  API_BEGIN
  if (L < 2 || k < 0 || k > L - 2 || !h || !v || nl < 1 || nr < 1 || !sec_l || !sec_r || !checked || !bad)
    throw Fail{DMRG_EINVAL, "dmrg_debug_validate: bad arguments"};
  ChainTune T;
  if (tune) {
    if (!(tune[0] >= 1.0) || !(tune[1] >= 0.0) || tune[2] < 1 || tune[2] > 129 || (tune[3] != 0 && tune[3] != 1) ||
        (tune[4] != 0 && tune[4] != 1))
      throw Fail{DMRG_EINVAL, "dmrg_debug_validate: bad tune"};
    T.target_chunks = tune[0];
    T.min_chunk = tune[1];
    T.tc_min = (int)tune[2];
    T.by_work = (int)tune[3];
    T.tc_tiny = (int)tune[4];
  }
  if (std::abs(two_sz) > N || ((N - two_sz) & 1)) throw Fail{DMRG_EINVAL, "two_sz incompatible with N"};
  Integrals I;
  I.L = L;
  I.h.assign(h, h + (size_t)L * L);
  I.v.assign(v, v + (size_t)L * L * L * L);
  auto sectors = [](int n, const int *t) {
    std::vector<Sector> out;
    for (int i = 0; i < n; ++i) out.push_back({t[3 * i], t[3 * i + 1], t[3 * i + 2]});
    return out;
  };
  std::vector<int> ls, rs;
  for (int s = 0; s < k; ++s) ls.push_back(s);
  for (int s = k + 2; s < L; ++s) rs.push_back(s);
  BlockLayout lb, rb;
  build_layout(lb, 0, L, ls, sectors(nl, sec_l));
  build_layout(rb, 1, L, rs, sectors(nr, sec_r));
  Psi Y = psi_layout(lb, rb, (N + two_sz) / 2, (N - two_sz) / 2);
  TempSet temps;
  auto rps = resolve_pieces(I, k, lb, rb, temps);
  const BlockLayout *lay[2] = {&lb, &rb};
  temps.layout(lay);
  // four operand arenas at distinct, far-apart element bases, so that every
  // operand address names its arena
  const uint64_t base[4] = {1ull << 40, 1ull << 41, 1ull << 42, 1ull << 43};
  const int64_t size[4] = {lb.total, rb.total, temps.total[0], temps.total[1]};
  const void *ptr[4];
  for (int a = 0; a < 4; ++a) ptr[a] = reinterpret_cast<const void *>((uintptr_t)(base[a] * 8));
  Arenas A{{&lb, &rb}, {ptr[0], ptr[1]}, &temps, {ptr[2], ptr[3]}, 8};
  ChainList CL;
  double f = 0.0;
  expand_hpsi_grouped(rps, A, Y, lb, CL, f);
  ExecPlan X;
  plan_exec(CL, tensor_cores != 0, true, T, X);
  long long nchk = 0, nbad = 0;
  std::string first;
  auto view = [&](const char *what, uint64_t at, int rows, int cols, int rst, int cst, bool op) {
    ++nchk;
    if (rows < 1 || cols < 1 || rst < 0 || cst < 0) {
      if (!nbad++) first = std::string(what) + ": bad shape or stride";
      return;
    }
    const uint64_t last = at + (uint64_t)(rows - 1) * rst + (uint64_t)(cols - 1) * cst;
    uint64_t lo = 0, hi = (uint64_t)Y.dim;  // psi and slots are relative offsets
    if (op) {
      int a = -1;
      for (int i = 0; i < 4; ++i)
        if (at >= base[i]) a = i;
      if (a < 0) {
        if (!nbad++) first = std::string(what) + ": address outside every arena";
        return;
      }
      lo = base[a];
      hi = base[a] + (uint64_t)size[a];
    }
    if (at < lo || last >= hi)
      if (!nbad++) first = std::string(what) + ": view leaves its array";
  };
  const std::vector<ChainGroup> *kinds[3] = {&X.vb, &X.vf, &X.vt};
  for (const auto *kv : kinds)
    for (const ChainGroup &t : *kv) {
      ++nchk;
      const uint64_t slot_last = t.d + (uint64_t)(t.m - 1) * t.drs + (uint64_t)(t.q - 1) * t.dcs;
      if (t.m < 1 || t.q < 1 || slot_last >= (uint64_t)X.soff)
        if (!nbad++) first = "chunk slot leaves the scratch array";
      for (int i = t.first; i < t.first + t.count; ++i) {
        const ChainEntry &e = X.xs[(size_t)i];
        if (e.x == ~0ull) {
          if (e.n != t.m && !nbad++) first = "identity X is not square";
        } else {
          view("X", e.x, t.m, e.n, e.xrs, e.xcs, true);
        }
        view("Y", e.y, e.n, e.p, e.yrs, e.ycs, false);
        if (e.z == ~0ull) {
          if (e.p != t.q && !nbad++) first = "identity Z is not square";
        } else {
          view("Z", e.z, e.p, t.q, e.zrs, e.zcs, true);
        }
      }
    }
  for (const ReduceGroup &r : X.vr) {
    view("output block", r.d, r.m, r.q, r.drs, r.dcs, false);
    ++nchk;
    if (r.soff + (int64_t)r.nsplit * r.m * r.q > X.soff && !nbad++) first = "reduction slots leave the scratch array";
  }
  if (tensor_cores && !X.vt.empty()) {
    // the tensor-core plan: every tile's source view inside its arena (the plan keeps
    // FP32-element addresses times 4, here the synthetic arena bases above), every
    // tile and every task's tile reads inside the tile arenas
    TcPlan P;
    plan_tc(X.xs, X.vt, P, nullptr, 4, T.tc_tiny);
    auto c16 = [](int x) { return (uint64_t)((x + 15) & ~15); };
    for (const TileSpec &t : P.ts) {
      ++nchk;
      if (t.dst + c16(t.R) * c16(t.K) * 4 > P.opbytes && !nbad++) first = "operator tile leaves the tile arena";
      if (t.src != ~0ull) view("operator tile source", t.src / 4, t.R, t.K, t.rs, t.cs, true);
    }
    for (const PsiTileSpec &t : P.ps) {
      ++nchk;
      if (t.dst + c16(t.p) * c16(t.n) * 4 > P.psibytes && !nbad++) first = "psi tile leaves the tile arena";
      view("psi tile source", (uint64_t)t.src, t.n, t.p, t.p, 1, false);
    }
    for (size_t g = 0; g < P.tg.size(); ++g) {
      const TcGroup &G = P.tg[g];
      for (int i = G.first; i < G.first + G.count; ++i) {
        const TcEntry &e = P.te[(size_t)i];
        ++nchk;
        if ((e.xt + c16(G.m) * c16(e.n) * 4 > P.opbytes || e.zt + c16(G.q) * c16(e.p) * 4 > P.opbytes ||
             e.yt + c16(e.p) * c16(e.n) * 4 > P.psibytes || e.stack > 8 || i + e.stack > G.first + G.count) &&
            !nbad++)
          first = "tensor-core task reads outside its tiles or stack";
      }
      ++nchk;
      const uint64_t slot_last = G.d + (uint64_t)(G.m - 1) * G.drs + (uint64_t)(G.q - 1) * G.dcs;
      if (slot_last >= (uint64_t)X.soff && !nbad++) first = "tensor-core output slot leaves the scratch array";
    }
  }
  *checked = nchk;
  *bad = nbad;
  if (nbad) set_error("dmrg_debug_validate: " + first);
  API_END
}

extern "C" int dmrg_debug_tc(int L, int N, int two_sz, const double *h, const double *v, int k, int nl,
                             const int *sec_l, int nr, const int *sec_r, const double *tune, long long *counts,
                             long long *te_out, long long *tg_out, long long *ts_out, long long *ps_out) {
  API_BEGIN
  if (L < 2 || k < 0 || k > L - 2 || !h || !v || nl < 1 || nr < 1 || !sec_l || !sec_r || !counts)
    throw Fail{DMRG_EINVAL, "dmrg_debug_tc: bad arguments"};
  if (std::abs(two_sz) > N || ((N - two_sz) & 1)) throw Fail{DMRG_EINVAL, "two_sz incompatible with N"};
  ChainTune T;
  if (tune) {
    if (!(tune[0] >= 1.0) || !(tune[1] >= 0.0) || tune[2] < 1 || tune[2] > 129 || (tune[3] != 0 && tune[3] != 1) ||
        (tune[4] != 0 && tune[4] != 1))
      throw Fail{DMRG_EINVAL, "dmrg_debug_tc: bad launch-shape parameters"};
    T.target_chunks = tune[0];
    T.min_chunk = tune[1];
    T.tc_min = (int)tune[2];
    T.by_work = (int)tune[3];
    T.tc_tiny = (int)tune[4];
  }
  Integrals I;
  I.L = L;
  I.h.assign(h, h + (size_t)L * L);
  I.v.assign(v, v + (size_t)L * L * L * L);
  auto sectors = [](int n, const int *t) {
    std::vector<Sector> out;
    for (int i = 0; i < n; ++i) out.push_back({t[3 * i], t[3 * i + 1], t[3 * i + 2]});
    return out;
  };
  std::vector<int> ls, rs;
  for (int s = 0; s < k; ++s) ls.push_back(s);
  for (int s = k + 2; s < L; ++s) rs.push_back(s);
  BlockLayout lb, rb;
  build_layout(lb, 0, L, ls, sectors(nl, sec_l));
  build_layout(rb, 1, L, rs, sectors(nr, sec_r));
  Psi Y = psi_layout(lb, rb, (N + two_sz) / 2, (N - two_sz) / 2);
  TempSet temps;
  auto rps = resolve_pieces(I, k, lb, rb, temps);
  const BlockLayout *lay[2] = {&lb, &rb};
  temps.layout(lay);
  Arenas A{{&lb, &rb}, {nullptr, nullptr}, &temps, {nullptr, nullptr}, 4};  // FP32 operand addresses
  ChainList CL;
  double f = 0.0;
  expand_hpsi_grouped(rps, A, Y, lb, CL, f);
  ExecPlan X;
  plan_exec(CL, true, true, T, X);
  TcPlan P;
  std::vector<int> src;
  plan_tc(X.xs, X.vt, P, &src, 4, T.tc_tiny);
  counts[0] = (long long)P.te.size();
  counts[1] = (long long)P.tg.size();
  counts[2] = (long long)P.ts.size();
  counts[3] = (long long)P.ps.size();
  counts[4] = (long long)P.opbytes;
  counts[5] = (long long)P.psibytes;
  counts[6] = P.ntc_shape[2];
  counts[7] = P.ntc_shape[1];
  counts[8] = P.ntc_shape[0];
  if (te_out)
    for (size_t i = 0; i < P.te.size(); ++i) {
      const TcEntry &t = P.te[i];
      const ChainEntry &e = X.xs[(size_t)src[i]];
      long long *o = te_out + 14 * i;
      const long long v14[14] = {(long long)t.xt, (long long)t.yt, (long long)t.zt, t.stack, src[i],
                                 (long long)e.x, e.xrs, e.xcs, (long long)e.z, e.zrs, e.zcs,
                                 (long long)e.y, t.n, t.p};
      for (int j = 0; j < 14; ++j) o[j] = v14[j];
    }
  if (tg_out)
    for (size_t i = 0; i < P.tg.size(); ++i) {
      const TcGroup &g = P.tg[i];
      const long long v7[7] = {(long long)g.d, g.drs, g.dcs, g.m, g.q, g.first, g.count};
      for (int j = 0; j < 7; ++j) tg_out[7 * i + j] = v7[j];
    }
  if (ts_out)
    for (size_t i = 0; i < P.ts.size(); ++i) {
      const TileSpec &t = P.ts[i];
      const long long v6[6] = {(long long)t.src, (long long)t.dst, t.rs, t.cs, t.R, t.K};
      for (int j = 0; j < 6; ++j) ts_out[6 * i + j] = v6[j];
    }
  if (ps_out)
    for (size_t i = 0; i < P.ps.size(); ++i) {
      const PsiTileSpec &t = P.ps[i];
      const long long v4[4] = {(long long)t.src, (long long)t.dst, t.n, t.p};
      for (int j = 0; j < 4; ++j) ps_out[4 * i + j] = v4[j];
    }
  API_END
}

extern "C" int dmrg_selftest_tcgen05(int N, int K, const float *A, const float *B, float *C) {
  API_BEGIN
  if (!A || !B || !C || N < 16 || N > 256 || N % 16 || K < 16 || K > 64 || K % 16)
    throw Fail{DMRG_EINVAL, "dmrg_selftest_tcgen05: N in 16..256, K in 16..64, multiples of 16"};
  DBuf<float> a, b, cc;
  DBuf<int> st;
  a.alloc(128 * K);
  b.alloc((size_t)N * K);
  cc.alloc((size_t)128 * N);
  st.alloc(1);
  CK(cudaMemcpy(a.p, A, 128 * K * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b.p, B, (size_t)N * K * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemset(st.p, 0, sizeof(int)));
  CK(launch_tc_selftest(a.p, b.p, cc.p, N, K, st.p, nullptr));
  CK(cudaDeviceSynchronize());
  int status = 0;
  CK(cudaMemcpy(&status, st.p, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(C, cc.p, (size_t)128 * N * sizeof(float), cudaMemcpyDeviceToHost));
  if (status) throw Fail{DMRG_ETIMEOUT, "tcgen05 self-test: mbarrier wait ran out"};
  API_END
}

// ---------------------------------------------------------------------------
// H.psi without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need H.psi:
// applications that reserve their whole device-memory budget up front and
// hand out no more afterwards, or code on a latency-critical path that must
// not block on the CUDA allocator.  dmrg_hpsi_noalloc serves them: the chunk
// partials of the split task list live in a fixed file-scope device array
// instead of memory allocated per plan.  The array is shared by every call and
// every context in the process and keeps the last call's contents; the call
// clears the part it uses first.  Calls whose kernels overlap on the GPU
// (other streams, other host threads) race on it, so such callers must
// order their calls on one stream or serialize them.
// ---------------------------------------------------------------------------
static constexpr long long kNoAllocScratchDoubles = 1ll << 21;  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
static std::mutex g_noalloc_mu;
static std::map<int, double *> g_noalloc_addr;  // device ordinal -> address of the array

// Device address of the array on the current device, looked up once per device.
// Host code must not use &g_noalloc_scratch itself: on the host that name is a
// stand-in, not a device address.
static double *noalloc_scratch() {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it != g_noalloc_addr.end()) return it->second;
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    throw Fail{DMRG_ECUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") + cudaGetErrorString(e)};
  g_noalloc_addr[dev] = static_cast<double *>(p);
  return static_cast<double *>(p);
}

extern "C" long long dmrg_hpsi_noalloc_capacity(void) { return kNoAllocScratchDoubles; }

extern "C" int dmrg_check_status(dmrg_ctx *c) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "ctx is NULL"};
  check_status(c);
  API_END
}

extern "C" int dmrg_debug_set_wait_limit(long long tries) {
  set_tc_wait_tries(tries);
  return DMRG_OK;
}

extern "C" int dmrg_debug_fail_alloc(long long n) {
  g_fail_alloc_after.store(n > 0 ? n : 0);
  return DMRG_OK;
}

extern "C" int dmrg_hpsi_noalloc(dmrg_ctx *c, const double *psi, double *sigma) {
  API_BEGIN
  if (!c || !psi || !sigma) throw Fail{DMRG_EINVAL, "NULL argument"};
  HPlan &P = c->plan;
  if (!P.valid || P.k != c->k || P.lb != lblock(c) || P.rb != rblock(c))
    throw Fail{DMRG_ESTATE, "dmrg_hpsi_noalloc needs the H.psi task list of the current position; "
                            "call dmrg_hpsi or dmrg_hpsi_flops once at this position first"};
  const bool lowp = P.lowp;
  const DevChain &ch = lowp ? P.chain32 : P.chain;
  if (!ch.split) throw Fail{DMRG_ESTATE, "H.psi task list has no split partials"};
  if (ch.scratch_n > kNoAllocScratchDoubles)
    throw Fail{DMRG_EINVAL, "this position needs " + std::to_string(ch.scratch_n) +
                                " doubles of H.psi scratch; the no-allocation scratch holds " +
                                std::to_string(kNoAllocScratchDoubles) + " (use dmrg_hpsi)"};
  double *scratch = noalloc_scratch();
  // a time-out left by an earlier call is not this call's: clear the status word
  // (a time-out of this call is read by dmrg_check_status or the next synchronizing call)
  CK(cudaMemsetAsync(c->dstatus.p, 0, 8 * sizeof(int), c->stream));
  CK(cudaMemsetAsync(sigma, 0, P.psi.dim * sizeof(double), c->stream));
  ch.launch(0, (uint64_t)(uintptr_t)psi, 0, (uint64_t)(uintptr_t)sigma, c->stream, c->dstatus.p, scratch);
  API_END
}

// ---------------------------------------------------------------------------
// Batched independent instances (many small problems of uneven L and M): the
// H.psi task lists of all instances, each at its current position, are
// concatenated into one task list over one concatenated psi / sigma, so each
// kernel class runs as a single grouped launch for every instance; the launch
// sequence is captured once into a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct dmrg_batch {
  std::vector<dmrg_ctx *> ctx;
  std::vector<long long> gen;  // each context's plan generation when the batch was built
  std::vector<long long> off;  // n + 1 offsets into the concatenated vectors
  cudaStream_t stream = nullptr;
  bool lowp = false, tc = false;
  dmrg::ChainTune tune;
  DevChain chain;
  DBuf<double> psi, sigma;
  double flops = 0.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;
  // the graph runs on a private non-blocking stream (the legacy default stream
  // cannot be captured), ordered after and before the contexts' stream by events
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ~dmrg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (own) cudaStreamDestroy(own);
  }
};

// The concatenated task list of the batch: every context's H.psi list (at its
// current position) with psi / sigma offsets shifted by the context's offset.
static void batch_chainlist(const std::vector<dmrg_ctx *> &ctxs, ChainList &CL, std::vector<long long> &off,
                            double &flops) {
  off.assign(1, 0);
  flops = 0.0;
  for (dmrg_ctx *c : ctxs) {
    build_hplan(c);
    const HPlan &P = c->plan;
    const DevChain &src = P.lowp ? P.chain32 : P.chain;
    std::vector<ChainEntry> ent((size_t)src.nent);
    std::vector<ChainGroup> grp((size_t)src.nall);
    if (!ent.empty()) CK(cudaMemcpy(ent.data(), src.ent.p, ent.size() * sizeof(ChainEntry), cudaMemcpyDeviceToHost));
    if (!grp.empty()) CK(cudaMemcpy(grp.data(), src.all.p, grp.size() * sizeof(ChainGroup), cudaMemcpyDeviceToHost));
    const long long o = off.back();
    const int base = (int)CL.flat.size();
    for (auto e : ent) {
      e.y += (uint64_t)o;
      CL.flat.push_back(e);
    }
    for (auto g : grp) {
      g.d += (uint64_t)o;
      g.first += base;
      CL.grp.push_back(g);
    }
    off.push_back(o + P.psi.dim);
    flops += P.flops;
  }
}

extern "C" int dmrg_batch_create(int n, dmrg_ctx *const *ctxs, dmrg_batch **out) {
  API_BEGIN
  if (n < 1 || !ctxs || !out) throw Fail{DMRG_EINVAL, "bad arguments"};
  *out = nullptr;
  auto b = std::make_unique<dmrg_batch>();
  b->stream = ctxs[0]->stream;
  for (int i = 0; i < n; ++i) {
    dmrg_ctx *c = ctxs[i];
    if (!c) throw Fail{DMRG_EINVAL, "NULL context in batch"};
    if (c->stream != b->stream) throw Fail{DMRG_EINVAL, "batched contexts must share one stream"};
    if ((c->prec != DMRG_PREC_FP64) != (ctxs[0]->prec != DMRG_PREC_FP64))
      throw Fail{DMRG_EINVAL, "batched contexts must share the working precision class"};
    b->ctx.push_back(c);
  }
  ChainList CL;
  batch_chainlist(b->ctx, CL, b->off, b->flops);
  for (dmrg_ctx *c : b->ctx) b->gen.push_back(c->plan_gen);
  b->lowp = ctxs[0]->prec != DMRG_PREC_FP64;
  b->tc = ctxs[0]->prec == DMRG_PREC_BF16X3;
  b->chain.upload(CL, b->stream, b->tc, true, b->tune, ctxs[0]->prec == DMRG_PREC_FP32);
  b->psi.alloc((size_t)std::max<long long>(b->off.back(), 1));
  b->sigma.alloc((size_t)std::max<long long>(b->off.back(), 1));
  CK(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  CK(cudaStreamSynchronize(b->stream));
  *out = b.release();
  API_END
}

extern "C" int dmrg_batch_free(dmrg_batch *b) {
  if (!b) return DMRG_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  delete b;
  return DMRG_OK;
}

extern "C" int dmrg_batch_layout(dmrg_batch *b, long long *offsets, double *flops) {
  API_BEGIN
  if (!b) throw Fail{DMRG_EINVAL, "batch is NULL"};
  if (offsets) std::copy(b->off.begin(), b->off.end(), offsets);
  if (flops) *flops = b->flops;
  API_END
}

extern "C" int dmrg_batch_hpsi(dmrg_batch *b, const double *psi, double *sigma, int device_ptrs) {
  API_BEGIN
  if (!b || !psi || !sigma) throw Fail{DMRG_EINVAL, "NULL argument"};
  // the batch's task list addresses its contexts' operator copies: refuse if any was rebuilt
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (!b->ctx[i]->plan.valid || b->ctx[i]->plan_gen != b->gen[i])
      throw Fail{DMRG_ESTATE, "a batched context changed position, precision or launch shape since "
                              "dmrg_batch_create (create the batch again)"};
  const int64_t n = b->off.back();
  cudaStream_t cs = b->stream, s = b->own;
  CK(cudaMemcpyAsync(b->psi.p, psi, n * sizeof(double),
                     device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, cs));
  CK(cudaEventRecord(b->ev_in, cs));
  CK(cudaStreamWaitEvent(s, b->ev_in, 0));
  int *status = b->ctx[0]->dstatus.p;
  auto body = [&]() {
    CK(cudaMemsetAsync(b->sigma.p, 0, n * sizeof(double), s));
    b->chain.launch(0, (uint64_t)(uintptr_t)b->psi.p, 0, (uint64_t)(uintptr_t)b->sigma.p, s, status);
  };
  if (!b->exec) {
    body();  // first call runs directly (and sets kernel attributes), then captures the sequence
    const long long before = kernel_launch_count();
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    body();
    CK(cudaStreamEndCapture(s, &b->graph));
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->graph_kernels = kernel_launch_count() - before;
    add_kernel_launches(-b->graph_kernels);  // captured, not launched
  } else {
    CK(cudaGraphLaunch(b->exec, s));
    add_kernel_launches(b->graph_kernels);
  }
  CK(cudaEventRecord(b->ev_out, s));
  CK(cudaStreamWaitEvent(cs, b->ev_out, 0));
  CK(cudaMemcpyAsync(sigma, b->sigma.p, n * sizeof(double),
                     device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, cs));
  if (!device_ptrs) CK(cudaStreamSynchronize(cs));
  check_status(b->ctx[0]);
  API_END
}

// ---------------------------------------------------------------------------
// Autotuning of the launch shape of H.psi task lists (split granularity and
// tensor-core routing): each candidate task list is built and its complete
// launch sequence (zeroing, kernels, ordered reduction) timed with CUDA events
// on the caller's stream; the fastest is kept.  Results are identical up to
// floating-point summation order across candidates.
// ---------------------------------------------------------------------------

namespace dmrg {

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

static double time_chain(const DevChain &ch, const double *x, double *y, int64_t n,
                         cudaStream_t s, int *status, int reps) {
  EventPair ev;
  auto once = [&]() {
    CK(cudaMemsetAsync(y, 0, (size_t)n * sizeof(double), s));
    ch.launch(0, (uint64_t)(uintptr_t)x, 0, (uint64_t)(uintptr_t)y, s, status);
  };
  once();
  CK(cudaEventRecord(ev.a, s));
  for (int r = 0; r < reps; ++r) once();
  CK(cudaEventRecord(ev.b, s));
  CK(cudaEventSynchronize(ev.b));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ev.a, ev.b));
  return (double)ms / reps;
}

// Coordinate search: split granularity first, then (tensor cores only) the
// smallest output-block side routed to the tensor-core kernel.
static ChainTune autotune_chain(const ChainList &CL, bool tc, bool ops32, const double *x, double *y, int64_t n,
                                cudaStream_t s, int *status, int reps, ChainTune start, double &best_ms) {
  auto run = [&](const ChainTune &t) {
    DevChain ch;
    ch.upload(CL, s, tc, true, t, ops32);
    return time_chain(ch, x, y, n, s, status, reps);
  };
  ChainTune best = start;
  best_ms = run(best);
  const double targets[] = {2048.0, 8192.0, 32768.0, 131072.0};
  const double mins[] = {5.0e4, 2.0e5};
  for (double tg : targets)
    for (double mn : mins) {
      ChainTune t = best;
      t.target_chunks = tg;
      t.min_chunk = mn;
      if (t.target_chunks == best.target_chunks && t.min_chunk == best.min_chunk) continue;
      const double ms = run(t);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  for (int flip = 0; flip < 2; ++flip) {
    ChainTune t = best;
    if (flip == 0) t.by_work = 1 - best.by_work;
    else t.flat_wide = 1 - best.flat_wide;
    const double ms = run(t);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  if (tc) {
    ChainTune t = best;
    t.tc_tiny = 1 - best.tc_tiny;
    const double ms = run(t);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
    const int tcs[] = {1, 9, 17, 33, 49, 65};
    for (int v : tcs) {
      if (v == best.tc_min) continue;
      ChainTune t = best;
      t.tc_min = v;
      const double ms = run(t);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  }
  return best;
}

static void tune_out(const ChainTune &t, double *params) {
  if (!params) return;
  params[0] = t.target_chunks;
  params[1] = t.min_chunk;
  params[2] = t.tc_min;
  params[3] = t.by_work;
  params[4] = t.flat_wide;
  params[5] = t.tc_tiny;
}

}  // namespace dmrg

extern "C" int dmrg_autotune(dmrg_ctx *c, int reps, double *best_ms, double *params) {
  API_BEGIN
  if (!c || reps < 1) throw Fail{DMRG_EINVAL, "dmrg_autotune: NULL context or reps < 1"};
  build_hplan(c);
  HPlan &P = c->plan;
  const bool lowp = P.lowp, tc = c->prec == DMRG_PREC_BF16X3;
  const int64_t n = P.psi.dim;
  ChainTune best;
  double ms = 0.0;
  {
    ChainList CL;
    double fl = 0.0;
    hpsi_chainlist(c, c->prec == DMRG_PREC_FP32, CL, fl);
    DBuf<double> x, y;
    x.alloc((size_t)std::max<int64_t>(n, 1));
    y.alloc((size_t)std::max<int64_t>(n, 1));
    CK(launch_fill_guess(x.p, n, 0x5eedull, c->stream));
    best = autotune_chain(CL, tc, c->prec == DMRG_PREC_FP32, x.p, y.p, n, c->stream, c->dstatus.p, reps, c->tune,
                          ms);
    CK(cudaStreamSynchronize(c->stream));
  }
  check_status(c);
  c->tune = best;
  c->plan.valid = false;  // rebuilt with the chosen shape
  build_hplan(c);
  if (best_ms) *best_ms = ms;
  tune_out(best, params);
  API_END
}

extern "C" int dmrg_set_tune(dmrg_ctx *c, double target_chunks, double min_chunk, int tc_min, int by_work,
                             int flat_wide, int tc_tiny) {
  API_BEGIN
  if (!c || !(target_chunks >= 1.0) || !(min_chunk >= 0.0) || tc_min < 1 || tc_min > 129 ||
      (by_work != 0 && by_work != 1) || (flat_wide != 0 && flat_wide != 1) || (tc_tiny != 0 && tc_tiny != 1))
    throw Fail{DMRG_EINVAL, "dmrg_set_tune: target_chunks >= 1, min_chunk >= 0, 1 <= tc_min <= 129, "
                            "by_work, flat_wide and tc_tiny 0 or 1"};
  c->tune.flat_wide = flat_wide;
  c->tune.tc_tiny = tc_tiny;
  c->tune.target_chunks = target_chunks;
  c->tune.min_chunk = min_chunk;
  c->tune.tc_min = tc_min;
  c->tune.by_work = by_work;
  c->plan.valid = false;
  API_END
}

extern "C" int dmrg_set_renorm_precision(dmrg_ctx *c, int precision) {
  API_BEGIN
  if (!c || (precision != DMRG_PREC_FP64 && precision != DMRG_PREC_FP32))
    throw Fail{DMRG_EINVAL, "dmrg_set_renorm_precision: NULL context or precision not FP64 / FP32"};
  c->renorm_prec = precision;
  API_END
}

extern "C" int dmrg_set_davidson(dmrg_ctx *c, int refine_keep, int sweep_max_iter) {
  API_BEGIN
  if (!c || refine_keep < 0 || refine_keep > 8 || sweep_max_iter < 1)
    throw Fail{DMRG_EINVAL, "dmrg_set_davidson: NULL context, refine_keep outside 0..8 or sweep_max_iter < 1"};
  c->refine_keep = refine_keep;
  c->sweep_max_iter = sweep_max_iter;
  API_END
}

extern "C" int dmrg_truncation_stats(dmrg_ctx *c, double *last_gap, double *min_gap,
                                     long long *truncations, long long *straddled) {
  API_BEGIN
  if (!c) throw Fail{DMRG_EINVAL, "NULL context"};
  if (last_gap) *last_gap = c->cut_gap;
  if (min_gap) *min_gap = c->min_cut_gap;
  if (truncations) *truncations = c->truncations;
  if (straddled) *straddled = c->straddled;
  API_END
}

extern "C" int dmrg_block_basis(dmrg_ctx *c, int side, int sites, int *nsec, int *kept, double *O,
                                long long *nO) {
  API_BEGIN
  if (!c || (side != 0 && side != 1) || sites < 1) throw Fail{DMRG_EINVAL, "dmrg_block_basis: bad arguments"};
  const auto &store = side == 0 ? c->left : c->right;
  const DevBlock *b = sites < (int)store.size() ? store[(size_t)sites].get() : nullptr;
  if (!b || b->parent.empty() || b->kept.size() != b->parent.size())
    throw Fail{DMRG_ESTATE, "dmrg_block_basis: no stored basis for that block"};
  int64_t total = 0;
  for (size_t e = 0; e < b->parent.size(); ++e) total += (int64_t)b->parent[e].dim * b->kept[e];
  if (nsec) *nsec = (int)b->parent.size();
  if (nO) *nO = (long long)total;
  if (kept)
    for (size_t e = 0; e < b->kept.size(); ++e) kept[e] = b->kept[e];
  if (O && total > 0) {
    if (!b->O.p || b->O.n < (size_t)total) throw Fail{DMRG_ESTATE, "dmrg_block_basis: basis not resident"};
    CK(cudaMemcpyAsync(O, b->O.p, (size_t)total * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  API_END
}

static void current_entropies(dmrg_ctx *c, double s3[3], double *rho2) {
  if (!c->psi_valid) throw Fail{DMRG_ESTATE, "no wave function at this position"};
  require_blocks(c);
  const Psi Y = psi_layout(lblock(c)->lay, rblock(c)->lay, c->nu, c->nd);
  if ((size_t)Y.dim > c->psi.n) throw Fail{DMRG_ESTATE, "wave function does not match the position's layout"};
  std::vector<double> h((size_t)std::max<int64_t>(Y.dim, 1));
  CK(cudaMemcpyAsync(h.data(), c->psi.p, Y.dim * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<PsiBlockRef> blocks;
  for (const PsiBlock &b : Y.blk) blocks.push_back({b.a, b.b, b.c, b.d, b.off, (int64_t)b.ma * b.md});
  double rho[256];
  pair_rdm(blocks, h.data(), rho);
  if (rho2)
    for (int i = 0; i < 256; ++i) rho2[i] = rho[i];
  if (s3) orbital_entropies(rho, s3);
}

// ---------------------------------------------------------------- orbital mutual information

// Two-orbital reduced density matrices of every orbital pair, for the orbital
// ordering of Sec. 3 (mutual information I_ij = s_i + s_j - s_ij), from the
// wave function at position 0 and the right blocks of sites 2..L-1 as stored:
// each right block state is a column of its renormalization matrix over
// (site state) x (next right block state), and those columns are orthonormal,
// so tracing every site right of the second orbital is the identity.  Working
// from site 0 to the right, a density matrix over the current right block with
// the first orbital's states left open (V) is carried through the sites
// between the two orbitals, each traced, and closed at the second orbital.
// Fermionic signs: the pair's matrix is that of the two orbitals moved next to
// each other in the Jordan-Wigner order (lattice order, up before down), so an
// element that changes the parity of the pair's first orbital picks up
// (-1)^(particles of each traced site between the two).
namespace {
struct HostExp {  // a right block's states over (site state s) x (next block state y)
  struct Piece {
    int s, y, my;
    const double *P;  // my x dim(new sector) rows of the block's O, row stride = dim(new sector)
  };
  std::vector<int> dim;
  std::vector<std::vector<Piece>> pieces;  // per new sector
  std::vector<double> O;
};
using SecMat = std::map<std::pair<int, int>, std::vector<double>>;  // (ket sector, bra sector) -> dense
}  // namespace

static void host_expansion(const DevBlock &b, cudaStream_t s, HostExp &X) {
  X.O.resize(b.O.n);
  if (b.O.n) CK(cudaMemcpyAsync(X.O.data(), b.O.p, b.O.n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  X.dim.clear();
  X.pieces.clear();
  for (size_t e = 0; e < b.parent.size(); ++e) {
    const int ma = b.kept[e];
    if (ma <= 0) continue;
    X.dim.push_back(ma);
    std::vector<HostExp::Piece> ps;
    for (const ESub &sb : b.parent[e].sub)
      ps.push_back({sb.x, sb.y, sb.m, X.O.data() + b.Ooff[e] + (int64_t)sb.roff * ma});
    X.pieces.push_back(ps);
  }
}

// C (m x n) += alpha * A (m x k, row stride lda) * op(B); B is k x n (row stride ldb) or, with
// bt, n x k read transposed
static void hgemm(double *C, const double *A, int lda, const double *B, int ldb, int m, int n, int k, bool bt,
                  double alpha) {
  for (int i = 0; i < m; ++i)
    for (int p = 0; p < k; ++p) {
      const double a = alpha * A[(int64_t)i * lda + p];
      if (a == 0.0) continue;
      double *c = C + (int64_t)i * n;
      if (bt)
        for (int j = 0; j < n; ++j) c[j] += a * B[(int64_t)j * ldb + p];
      else
        for (int j = 0; j < n; ++j) c[j] += a * B[(int64_t)p * ldb + j];
    }
}

// out[(y, y')] += sgn * P_{A,s,y} V[(A, A')] P_{A',s',y'}^T over pieces with (s, s') accepted by keep
template <class Keep>
static void mi_expand(const HostExp &X, const SecMat &V, SecMat &out, const std::vector<int> &ydim, Keep keep) {
  for (const auto &kv : V) {
    const int A = kv.first.first, A2 = kv.first.second;
    const int da = X.dim[A], da2 = X.dim[A2];
    for (const auto &p : X.pieces[A]) {
      std::vector<double> T;
      bool have_t = false;
      for (const auto &q : X.pieces[A2]) {
        double w;
        if (!keep(p.s, q.s, w)) continue;
        if (!have_t) {  // T = P_p V (my x da2)
          T.assign((size_t)p.my * da2, 0.0);
          hgemm(T.data(), p.P, da, kv.second.data(), da2, p.my, da2, da, false, 1.0);
          have_t = true;
        }
        auto &o = out[{p.y, q.y}];
        if (o.empty()) o.assign((size_t)ydim[p.y] * ydim[q.y], 0.0);
        hgemm(o.data(), T.data(), da2, q.P, da2, p.my, q.my, da2, true, w);
      }
    }
  }
}

// rho[s][s'] += tr_y(P_{A,s,y} V[(A, A')] P_{A',s',y}^T): the second orbital opened, the rest traced
static void mi_close(const HostExp &X, const SecMat &V, double rho[4][4]) {
  for (const auto &kv : V) {
    const int A = kv.first.first, A2 = kv.first.second;
    const int da = X.dim[A], da2 = X.dim[A2];
    for (const auto &p : X.pieces[A])
      for (const auto &q : X.pieces[A2]) {
        if (p.y != q.y) continue;
        std::vector<double> T((size_t)p.my * da2, 0.0);
        hgemm(T.data(), p.P, da, kv.second.data(), da2, p.my, da2, da, false, 1.0);
        double t = 0.0;
        for (int r = 0; r < p.my; ++r)
          for (int c2 = 0; c2 < da2; ++c2) t += T[(size_t)r * da2 + c2] * q.P[(int64_t)r * da2 + c2];
        rho[p.s][q.s] += t;
      }
  }
}

static int site_n(int s) { return SITE_NU[s] + SITE_ND[s]; }

static void mutual_information(dmrg_ctx *c, double *I, double *s1, double *rho_all) {
  const int L = c->L;
  if (c->k != 0) throw Fail{DMRG_ESTATE, "mutual information needs the wave function at position 0"};
  if (!c->psi_valid) throw Fail{DMRG_ESTATE, "no wave function at position 0 (run dmrg_davidson)"};
  require_blocks(c);
  for (int n = 1; n <= L - 2; ++n)
    if (n >= (int)c->right.size() || !c->right[n] || c->right[n]->parent.empty())
      throw Fail{DMRG_ESTATE, "mutual information needs the right blocks of every length (one backward pass)"};
  const Psi Y = psi_layout(lblock(c)->lay, rblock(c)->lay, c->nu, c->nd);
  std::vector<double> h((size_t)std::max<int64_t>(Y.dim, 1));
  CK(cudaMemcpyAsync(h.data(), c->psi.p, Y.dim * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // R_m = right block of sites m..L-1 = c->right[L - m]
  std::vector<HostExp> X((size_t)L + 1);
  std::vector<std::vector<int>> dims((size_t)L + 1);
  for (int m = 2; m <= L; ++m) {
    const DevBlock &b = *c->right[L - m];
    for (const auto &sec : b.lay.sec) dims[m].push_back(sec.dim);
    if (m < L) host_expansion(b, c->stream, X[m]);
  }
  std::vector<double> R((size_t)L * L * 256, 0.0);  // rho of pair (i, j), i < j
  auto pair_rho = [&](int i, int j) { return R.data() + ((size_t)i * L + j) * 256; };
  // pair (0, 1): the two sites of position 0
  {
    std::vector<PsiBlockRef> blocks;
    for (const PsiBlock &b : Y.blk) blocks.push_back({b.a, b.b, b.c, b.d, b.off, (int64_t)b.ma * b.md});
    pair_rdm(blocks, h.data(), pair_rho(0, 1));
  }
  // carry V (first orbital i open) from R_m to the right end
  auto run = [&](int i, int m, std::array<SecMat, 16> V) {
    for (int j = m; j <= L - 1; ++j) {
      for (int sg = 0; sg < 16; ++sg) {
        double rr[4][4] = {};
        mi_close(X[j], V[sg], rr);
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) pair_rho(i, j)[(4 * (sg / 4) + a) * 16 + 4 * (sg % 4) + b] += rr[a][b];
      }
      if (j == L - 1) break;
      for (int sg = 0; sg < 16; ++sg) {
        const bool odd = (site_n(sg / 4) + site_n(sg % 4)) & 1;
        SecMat nv;
        mi_expand(X[j], V[sg], nv, dims[j + 1], [&](int s, int s2, double &w) {
          w = (odd && (site_n(s) & 1)) ? -1.0 : 1.0;
          return s == s2;
        });
        V[sg].swap(nv);
      }
    }
  };
  auto vec = [&](const PsiBlock &b) { return h.data() + b.off; };
  // first orbital 0 (site 1 traced, with the string sign) and 1 (site 0 traced)
  for (int i = 0; i < 2 && L > 2; ++i) {
    std::array<SecMat, 16> V;
    for (const PsiBlock &p : Y.blk)
      for (const PsiBlock &q : Y.blk) {
        const int sp = i == 0 ? p.b : p.c, sq = i == 0 ? q.b : q.c;  // open states
        const int tp = i == 0 ? p.c : p.b, tq = i == 0 ? q.c : q.b;  // traced states
        if (tp != tq) continue;
        const bool odd = (site_n(sp) + site_n(sq)) & 1;
        const double w = (i == 0 && odd && (site_n(tp) & 1)) ? -1.0 : 1.0;
        auto &o = V[4 * sp + sq][{p.d, q.d}];
        if (o.empty()) o.assign((size_t)p.md * q.md, 0.0);
        hgemm(o.data(), vec(p), 1, vec(q), q.md, p.md, q.md, 1, false, w);
      }
    run(i, 2, V);
  }
  // first orbital m >= 2: W (everything left of m traced) over R_m, opened at m
  SecMat W;
  for (const PsiBlock &p : Y.blk)
    for (const PsiBlock &q : Y.blk) {
      if (p.b != q.b || p.c != q.c || p.d != q.d) continue;
      auto &o = W[{p.d, q.d}];
      if (o.empty()) o.assign((size_t)p.md * q.md, 0.0);
      hgemm(o.data(), vec(p), 1, vec(q), q.md, p.md, q.md, 1, false, 1.0);
    }
  for (int m = 2; m <= L - 2; ++m) {
    std::array<SecMat, 16> V;
    for (int sg = 0; sg < 16; ++sg)
      mi_expand(X[m], W, V[sg], dims[m + 1], [&](int s, int s2, double &w) {
        w = 1.0;
        return s == sg / 4 && s2 == sg % 4;
      });
    run(m, m + 1, V);
    SecMat nw;
    mi_expand(X[m], W, nw, dims[m + 1], [&](int s, int s2, double &w) {
      w = 1.0;
      return s == s2;
    });
    W.swap(nw);
  }
  // entropies from the pair matrices
  std::vector<double> s1v((size_t)L, 0.0);
  if (I) std::fill(I, I + (size_t)L * L, 0.0);
  for (int i = 0; i < L; ++i)
    for (int j = i + 1; j < L; ++j) {
      double s3[3];
      orbital_entropies(pair_rho(i, j), s3);
      s1v[i] = s3[0];
      s1v[j] = s3[1];
      if (I) I[(size_t)i * L + j] = I[(size_t)j * L + i] = s3[0] + s3[1] - s3[2];
    }
  if (s1) std::copy(s1v.begin(), s1v.end(), s1);
  if (rho_all) std::copy(R.begin(), R.end(), rho_all);
}

extern "C" int dmrg_mutual_information(dmrg_ctx *c, double *I, double *s1, double *rho_pairs) {
  API_BEGIN
  if (!c || (!I && !s1 && !rho_pairs)) throw Fail{DMRG_EINVAL, "NULL argument"};
  if (c->L < 2) throw Fail{DMRG_EINVAL, "mutual information needs L >= 2"};
  mutual_information(c, I, s1, rho_pairs);
  API_END
}

extern "C" int dmrg_orbital_entropies(dmrg_ctx *c, double *s3, double *rho2) {
  API_BEGIN
  if (!c || (!s3 && !rho2)) throw Fail{DMRG_EINVAL, "NULL argument"};
  current_entropies(c, s3, rho2);
  API_END
}

extern "C" int dmrg_get_tune(dmrg_ctx *c, double *params) {
  API_BEGIN
  if (!c || !params) throw Fail{DMRG_EINVAL, "NULL argument"};
  tune_out(c->tune, params);
  API_END
}

extern "C" int dmrg_batch_autotune(dmrg_batch *b, int reps, double *best_ms, double *params) {
  API_BEGIN
  if (!b || reps < 1) throw Fail{DMRG_EINVAL, "dmrg_batch_autotune: NULL batch or reps < 1"};
  CK(cudaStreamSynchronize(b->stream));
  ChainList CL;
  std::vector<long long> off;
  double fl = 0.0;
  batch_chainlist(b->ctx, CL, off, fl);
  if (off != b->off) throw Fail{DMRG_ESTATE, "a batched context changed position since dmrg_batch_create"};
  b->gen.clear();
  for (dmrg_ctx *c : b->ctx) b->gen.push_back(c->plan_gen);
  const int64_t n = b->off.back();
  CK(launch_fill_guess(b->psi.p, n, 0x5eedull, b->stream));
  double ms = 0.0;
  ChainTune best = autotune_chain(CL, b->tc, b->ctx[0]->prec == DMRG_PREC_FP32, b->psi.p, b->sigma.p, n, b->stream,
                                  b->ctx[0]->dstatus.p, reps, b->tune, ms);
  check_status(b->ctx[0]);
  b->tune = best;
  b->chain.upload(CL, b->stream, b->tc, true, best, b->ctx[0]->prec == DMRG_PREC_FP32);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;  // captured again on the next dmrg_batch_hpsi
  CK(cudaStreamSynchronize(b->stream));
  if (best_ms) *best_ms = ms;
  tune_out(best, params);
  API_END
}
