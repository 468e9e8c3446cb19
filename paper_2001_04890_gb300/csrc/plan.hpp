// Host-side planner for the two-site QC-DMRG hot path (no CUDA in this file).
//
// Paper: Brabec et al., "Massively parallel quantum chemical density matrix
// renormalization group method", Sec. 2.1 (block / site / sector structure,
// pre-summed operators) and Sec. 2.2.1-2.2.3 (task lists for H.psi,
// renormalization and pre-summation).
//
// The planner turns the electronic Hamiltonian (Eq. H2q) into
//   * "pieces": products  l-op (x) s_l-op (x) s_r-op (x) r-op  of a block
//     operator of the left block, a 4x4 left-site matrix, a 4x4 right-site
//     matrix and a block operator of the right block (Eq. dgemm's
//     A_l (x) A_sl (x) A_sr (x) A_r, with the site factors kept as matrices);
//   * block operators that are stored (normal a+, a+a+, a+a; H; the
//     one-index complementary T / V) or formed on the fly as linear
//     combinations of stored ones (the pre-summed operators of Sec. 2.2.3,
//     Eq. presum);
// and then expands pieces over the sectors of Eq. wf_sec into the task list
// of Sec. 2.2.1 (one entry per (operator combination, s -> s')).
#pragma once

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdint>
#include <exception>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace dmrg {

// Run fn(i) for i in [0, n) on up to 16 host threads (work handed out one index
// at a time); the first exception of any worker is rethrown here.
template <class F>
inline void parallel_for(size_t n, F fn) {
  std::atomic<size_t> next{0};
  std::mutex err_mu;
  std::exception_ptr err;
  auto worker = [&]() {
    try {
      for (size_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) fn(i);
    } catch (...) {
      std::lock_guard<std::mutex> lk(err_mu);
      if (!err) err = std::current_exception();
      next.store(n);
    }
  };
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (unsigned t = 1; t < hw && t < n; ++t) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
  if (err) std::rethrow_exception(err);
}


using Mat4 = std::array<double, 16>;  // site matrix, row-major [b'][b]

// site state -> particle numbers (basis {0, up, dn, updn})
constexpr int SITE_NU[4] = {0, 1, 0, 1};
constexpr int SITE_ND[4] = {0, 0, 1, 1};

struct Integrals {
  int L = 0;
  std::vector<double> h;  // L*L
  std::vector<double> v;  // L^4 chemists' (ij|kl)
  // spin-orbital one-body t_pq and two-body w_pqrs = <pq|rs>
  double t(int p, int q) const {
    if ((p & 1) != (q & 1)) return 0.0;
    return h[(p >> 1) * L + (q >> 1)];
  }
  double w(int p, int q, int r, int s) const {
    if ((p & 1) != (r & 1) || (q & 1) != (s & 1)) return 0.0;
    const int64_t i = p >> 1, j = q >> 1, k = r >> 1, l = s >> 1;
    return v[((i * L + k) * L + j) * L + l];
  }
  double W(int p, int q, int r, int s) const { return w(p, q, r, s) - w(p, q, s, r); }
};

struct Sector {
  int nu, nd, dim;
};

// A stored operator family: operators with the same quantum-number change
// (dnu, dnd) on one block, laid out as [ket sector][k][bra row][ket col], so
// the K operators of one sector transition are adjacent in memory (the
// orbital-index leg of the operator tensors of Sec. 2.2, Fig. opclass).
struct Family {
  int kind = 0;      // KH, KC, KT, KV, KA, KB
  int dnu = 0, dnd = 0;
  std::vector<std::array<int, 2>> idx;  // per k: spin-orbital indices
  std::vector<int> bra;                 // per ket sector: bra sector or -1
  std::vector<int64_t> off;             // per ket sector: element offset of its slab
  int64_t size = 0;                     // elements
  int64_t base = 0;                     // element offset of the family in its arena
  int K() const { return (int)idx.size(); }
};

enum Kind { KH = 0, KC = 1, KT = 2, KV = 3, KA = 4, KB = 5 };

struct BlockLayout {
  int side = 0;                 // 0: left block, 1: right block
  int L = 0;
  std::vector<int> sites;       // ascending
  std::vector<Sector> sec;      // sorted by (nu, nd)
  std::vector<Family> fam;
  std::unordered_map<int64_t, std::pair<int, int>> lookup;  // (kind,i,j) -> (family, k)
  int64_t total = 0;            // elements of all families
  int find(int nu, int nd) const;
  bool empty() const { return sites.empty(); }
  bool has_site(int s) const;
  static int64_t key(int kind, int i, int j, int L) {
    return ((int64_t)kind * 4 * L + (i + 1)) * 4 * L + (j + 1);
  }
  bool get(int kind, int i, int j, int &f, int &k) const;
};

// Build the sector list, the stored families and their layout for a block.
void build_layout(BlockLayout &b, int side, int L, const std::vector<int> &sites,
                  const std::vector<Sector> &sec);

// A block-operator reference used inside pieces.
struct OpRef {
  int type = 0;   // 0 identity, 1 stored, 2 linear combination
  int kind = -1;  // stored kind / kind of all sources of a combination
  int i = -1, j = -1;
  bool tr = false;
  std::vector<std::tuple<int, int, double>> lc;  // (i, j, coef) for type 2
  int parity() const;                            // fermion parity of the operator
};

struct HalfPiece {
  OpRef blk;
  Mat4 site;
  double coef;
};
using HalfOp = std::vector<HalfPiece>;

struct Piece {
  double coef;
  OpRef l;
  Mat4 sl, sr;
  OpRef r;
  bool hc;  // add the Hermitian conjugate (transposed) contribution too
};

// Site matrices for one site (global site index s).
struct SiteAlgebra {
  const Integrals *I;
  Mat4 cdag(int p) const;  // c+_p, p a mode of this site
  Mat4 c(int p) const;
  Mat4 H(int s) const;
  Mat4 T(int s, int j) const;           // sum_i t_ij c+_i - sum_pqr w_pqrj c+_p c+_q c_r
  Mat4 V(int s, int i) const;           // sum_qrs w_iqrs c+_q c_s c_r
  Mat4 Pc(int s, int r, int q) const;   // sum_{a<b} W_ab,rq c+_a c+_b
  Mat4 Pa(int s, int p, int q) const;   // sum_{a<b} W_pq,ab c_b c_a
  Mat4 Q(int s, int p, int q) const;    // sum_ab (w_p a q b - w_p a b q) c+_a c_b
};

Mat4 mat_eye();
Mat4 mat_zero();
Mat4 mat_mul(const Mat4 &a, const Mat4 &b);
Mat4 mat_t(const Mat4 &a);
Mat4 mat_scale(const Mat4 &a, double s);
bool mat_is_zero(const Mat4 &a);
int mat_parity(const Mat4 &a);  // parity of a site matrix with definite quantum numbers

// Half operators of the enlarged left half L' = l u {sl} and right half
// R' = {sr} u r.  Left pieces are products (block op)(site op); right pieces
// are (site op)(block op).  k = position (sl = site k, sr = site k+1).
struct HalfOps {
  const Integrals *I;
  int L, k;
  int lsites, rfirst;  // l = [0, lsites), r = [rfirst, L)
  SiteAlgebra S;
  bool l_empty, r_empty;

  HalfOps(const Integrals *I_, int k_, bool l_empty_, bool r_empty_);
  int site_of(int p) const { return p >> 1; }
  bool in_l(int p) const { return site_of(p) < k; }
  bool is_sl(int p) const { return site_of(p) == k; }
  bool is_sr(int p) const { return site_of(p) == k + 1; }
  bool in_r(int p) const { return site_of(p) >= k + 2; }

  HalfOp L_I() const;
  HalfOp L_C(int p) const;
  HalfOp L_A(int p, int q) const;
  HalfOp L_B(int p, int s) const;
  HalfOp L_H() const;
  HalfOp L_T(int j) const;
  HalfOp L_Pc(int r, int s) const;
  HalfOp L_Q(int a, int b) const;

  HalfOp R_I() const;
  HalfOp R_C(int p) const;
  HalfOp R_c(int p) const;
  HalfOp R_A(int p, int q) const;
  HalfOp R_AT(int p, int q) const;
  HalfOp R_B(int p, int s) const;
  HalfOp R_H() const;
  HalfOp R_V(int i) const;
  HalfOp R_Pa(int p, int q) const;
  HalfOp R_Q(int a, int b) const;
};

// The pieces of H at position k (Sec. 2.2.1).
std::vector<Piece> hamiltonian_pieces(const Integrals &I, int k, bool l_empty, bool r_empty);

// Merge pieces that share one side exactly: sum_u X_u (x) S_u (x) Y = sum_E
// (sum_u S_u[E] X_u) (x) E (x) Y (a pre-summation, Sec. 2.2.3).
std::vector<Piece> compress_pieces(std::vector<Piece> in);

// For the renormalization of the new block (Sec. 2.2.2): the half operator
// defining each stored operator of the new block, in family order.
struct NewOp {
  int fam, k;
  HalfOp def;
};
std::vector<NewOp> new_block_ops(const Integrals &I, int k, int side, const BlockLayout &newb,
                                 bool old_empty);

// Text dump of pieces (for CPU-side checks of the term generation).
std::string dump_pieces(const std::vector<Piece> &ps);
std::string dump_halfop(const HalfOp &h);

// --------------------------------------------------------------------------
// resolved operators: stored family slices and pre-summed temporaries
// --------------------------------------------------------------------------

struct TempFamily {
  int side;       // block the sources live on (0 left, 1 right)
  int src_fam;    // source family
  bool tr;        // sources transposed
  int dnu, dnd;   // quantum-number change of the temporaries
  std::vector<std::vector<std::pair<int, double>>> coefs;  // per temp: (source k, coef)
  std::vector<int> bra;
  std::vector<int64_t> off;
  int64_t size = 0, base = 0;
  int K() const { return (int)coefs.size(); }
};

// An operator resolved to memory: identity, or (arena, family, k) with a
// transpose flag.  arena 0/1: stored families of the left/right block,
// arena 2/3: temporaries of the left/right block.
struct Ref {
  int arena = -1;
  int fam = -1, k = 0;
  bool tr = false;
  int dnu = 0, dnd = 0, par = 0;
};

// The sources of a linear-combination operator on a block, resolved to stored
// operators of one family, sorted, duplicates merged (prepare_temp: pure, so
// many can be prepared in parallel before TempSet numbers them in order).
struct PreparedTemp {
  bool zero = true;
  int fam = -1;
  std::vector<std::pair<int, double>> m;
  uint64_t hash = 0;
};
PreparedTemp prepare_temp(const BlockLayout &b, const OpRef &op);

struct TempSet {
  std::vector<TempFamily> fam[2];
  std::map<std::tuple<int, int, bool>, int> fam_of[2];
  std::unordered_map<uint64_t, std::vector<std::pair<int, int>>> dedup[2];  // hash -> (family, temp)
  int64_t total[2] = {0, 0};
  Ref make(int side, const BlockLayout &b, const OpRef &op, bool &zero);
  Ref make_prepared(int side, const BlockLayout &b, const OpRef &op, PreparedTemp &&pt, bool &zero);
  void layout(const BlockLayout *blocks[2]);
};

Ref resolve(const OpRef &op, int side, const BlockLayout &b, TempSet &temps, bool &zero);

// One entry of the batched triple product  D += f * X * Y * Z  used by H.psi,
// renormalization and the density matrix (addresses are element offsets
// relative to per-launch bases; identity operands have x or z == ~0).
struct ChainEntry {
  uint64_t x, y, z;
  int xrs, xcs, yrs, ycs, zrs, zcs;
  int n, p;
  double f;
};
struct ChainGroup {
  uint64_t d;
  int drs, dcs;
  int m, q;
  int first, count;
  int tile0;
};

// Launch-shape decisions of the task lists (pure host logic).

// Association of one task D += f X Y Z (X m x n, Y n x p, Z p x q): true when the
// transposed product D^T += f Z^T Y^T X^T (n p q + m n q multiply-adds) is
// strictly cheaper than (X Y) Z (m n p + m p q).
bool prefer_transposed(int m, int n, int p, int q);

// Stacks of a key list sorted so that equal keys are adjacent: the lengths of
// the runs of equal keys, each run cut into pieces of at most cap, in order.
std::vector<int> stack_runs(const std::vector<uint64_t> &sorted_keys, int cap);

// Truncation of the reduced density matrix (Sec. 2.1): keep the mkeep
// eigenvectors with the largest eigenvalues over all sectors.  Input: per sector,
// the eigenvalues in ascending order (as a symmetric eigensolver returns them).
// Order: descending eigenvalue, ties by (sector, in-sector rank from the top);
// eigenvalues <= drop are never kept.  When the mkeep-th and the next eigenvalue
// above drop differ by less than kTruncCluster, "the mkeep largest" is not
// defined: the cut moves down past that whole cluster (consecutive eigenvalues
// closer than kTruncCluster), so the kept space does not depend on how the
// cluster is split; only if nothing would be kept does the cut stay at mkeep.
// cols[e] lists the kept columns of sector e (indices into the ascending order)
// by descending eigenvalue.  cut_gap is the smallest kept eigenvalue minus the
// largest eigenvalue above drop that was not kept (+infinity when nothing above
// drop was cut, or nothing was kept): a gap below kTruncCluster remains only
// when the top cluster alone holds more than mkeep states.
constexpr double kTruncCluster = 1e-10;
struct KeptSet {
  std::vector<int> kept;
  std::vector<std::vector<int>> cols;
  double trace = 0.0, kept_weight = 0.0, cut_gap = 0.0;
};
KeptSet choose_kept(const std::vector<std::vector<double>> &ev_ascending, int mkeep, double drop);

// Orbital reduced density matrices of the two sites of a two-site wave function
// (Eq. wf_sec): block s = (a, b, c, d) holds psi_{a b c d} (m_a x m_d at psi +
// off, size = m_a m_d).  The two-orbital matrix over the site-state pairs
// 4 b + c is rho[(b c), (b' c')] = sum_{a,d} <psi_{a b c d}, psi_{a b' c' d}>
// (the local transition operators are parity-even, so no Jordan-Wigner sign
// enters); it is block diagonal in the pair's (n_up, n_dn).
struct PsiBlockRef {
  int a, b, c, d;
  int64_t off, size;
};
void pair_rdm(const std::vector<PsiBlockRef> &blocks, const double *psi, double rho[256]);
// Von Neumann entropies -sum x ln x of the trace-normalised one-orbital
// matrices of the left and right site (diagonal: the four site states differ
// in (n_up, n_dn)) and of the two-orbital matrix: out = {s_left, s_right, s_pair}.
void orbital_entropies(const double rho[256], double out[3]);
// Eigenvalues of a small symmetric matrix (n <= 16, row-major) by cyclic Jacobi rotations.
void small_symmetric_eigenvalues(int n, const double *a, double *ev);

}  // namespace dmrg
