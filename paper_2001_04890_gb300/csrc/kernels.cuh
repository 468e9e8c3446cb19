// Device kernels of the two-site QC-DMRG hot path (sm_103a) -- launch wrappers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "plan.hpp"

namespace dmrg {

// Pre-summation task (Sec. 2.2.3, Eq. presum): out[t] = sum_u coef[t,u] src[u]
// for the K_out temporaries of one family in one sector transition.
struct LincombTask {
  uint64_t out;        // element address of the output slab (K_out blocks)
  uint64_t src;        // element address of the source slab (K_src blocks)
  uint64_t coef;       // element address of the K_out x K_src coefficient matrix
  int kout, ksrc;
  int rows, cols;      // output block shape
  int tr;              // source blocks read transposed (source block is cols x rows)
  int tile0;           // first tile of this task in the launch grid
};

// Bounded-wait / error flag shared by the kernels of one context.
struct DevStatus {
  int error;
};

cudaError_t launch_chain_fp64(const ChainEntry *e, const ChainGroup *g, int ngroups, int ntiles,
                              uint64_t xb, uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s);
// same task list with FP32 operators X, Z (FP64 psi in, FP64 sigma out, FP32 accumulation)
cudaError_t launch_chain_f32ops(const ChainEntry *e, const ChainGroup *g, int ngroups, int ntiles,
                                uint64_t xb, uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s);
// one warp per output block of at most 32 x 32, lanes over flattened elements
// warps per CTA: FP64 6 or 4, FP32 12 or 8 (other values: the first)
cudaError_t launch_chain_flat_fp64(const ChainEntry *e, const ChainGroup *g, int ngroups, uint64_t xb,
                                   uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s, int warps = 6);
cudaError_t launch_chain_flat_f32ops(const ChainEntry *e, const ChainGroup *g, int ngroups, uint64_t xb,
                                     uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s, int warps = 12);

// Split task lists: every output block's entries are cut into chunks whose
// partial blocks go to a scratch buffer; this adds them in chunk order.
struct ReduceGroup {
  int64_t e0;    // first flattened element of this block among all reduced elements
  int64_t soff;  // scratch offset of chunk 0 (chunks are m*q apart)
  uint64_t d;    // element offset of the output block
  int drs, dcs, m, q, nsplit;
};
cudaError_t launch_reduce_partials(const ReduceGroup *r, int nred, int64_t total, const double *scratch,
                                   double *out, cudaStream_t s);
cudaError_t launch_to_f32(float *out, const double *in, int64_t n, cudaStream_t s);
cudaError_t launch_lincomb_fp64(const LincombTask *t, int ntasks, int ntiles, cudaStream_t s);
cudaError_t launch_diag_fp64(const ChainEntry *e, const ChainGroup *g, int ngroups,
                             uint64_t xb, uint64_t zb, double *diag, cudaStream_t s);

// Davidson helpers (all FP64, deterministic two-stage reductions)
cudaError_t launch_dots(const double *V, int k, int64_t n, const double *w, double *partial,
                        double *out, cudaStream_t s);
cudaError_t launch_combine(double *out, const double *V, const double *y, int k, int64_t n,
                           double beta, cudaStream_t s);
cudaError_t launch_axpy(double *y, const double *x, double a, int64_t n, cudaStream_t s);
cudaError_t launch_scale(double *x, const double *a_dev, int invert_sqrt, int64_t n, cudaStream_t s);
cudaError_t launch_precond(double *t, const double *r, const double *diag, const double *theta,
                           int64_t n, cudaStream_t s);
cudaError_t launch_residual(double *r, const double *hx, const double *x, const double *theta,
                            int64_t n, cudaStream_t s);
cudaError_t launch_sub_proj(double *w, const double *V, const double *c, int k, int64_t n,
                            cudaStream_t s);
cudaError_t launch_fill_guess(double *x, int64_t n, uint64_t seed, cudaStream_t s);
cudaError_t launch_jacobi_eigh(const double *A, int n, int lda, double *evals, double *evecs,
                               cudaStream_t s);
cudaError_t launch_gather_columns(double *O, const double *evecs, int n, const int *cols,
                                  int kept, cudaStream_t s);

int dots_partial_blocks(int64_t n);

// tcgen05 self-test: C (128 x N) = A (128 x K) B^T (N x K), bf16 inputs, FP32 accumulation in TMEM
cudaError_t launch_tc_selftest(const float *A, const float *B, float *C, int N, int K, int *status,
                               cudaStream_t s);

// number of kernels this library has launched in the process
long long kernel_launch_count();
void add_kernel_launches(long long n);  // kernels run by CUDA-graph replays

}  // namespace dmrg

namespace dmrg {

// Tensor-core tiles: an R x K operand pre-split into bf16 hi / lo parts in the
// K-major core-matrix layout (8-row x 16-byte core matrices, core matrix
// (rg, kg) at byte (rg * K16/8 + kg) * 128), rows padded to R8 = ceil8(R),
// K to K16 = ceil16(K) with zeros; the lo part follows the hi part.
struct TileSpec {
  uint64_t src;     // byte address of the source view (FP32 or FP64; element (r, k) at element r*rs + k*cs)
  uint64_t dst;     // byte offset of the tile in the tile arena
  int rs, cs, R, K;
};
struct PsiTileSpec {
  int64_t src;      // element offset of the psi block (n x p, row-major) in psi
  uint64_t dst;     // byte offset of its transposed tile (rows p, K n)
  int n, p;
};
// One task of the pipelined tensor-core chain: D += f X Y Z with X, Y^T, Z^T given as tiles.
// 32 bytes, so any run of entries is one aligned bulk copy.
struct TcEntry {
  uint64_t xt, zt;      // byte offsets of the X and Z^T tiles in the operator tile arena
  uint32_t yt;          // byte offset of the Y^T tile in the psi tile arena
  float f;
  uint8_t n, p;         // inner dims (<= 128)
  uint8_t stack;        // first task of a stack: the number of consecutive tasks (same Y, same
                        // output block) whose X run stacked along M in one stage 1; others 0
  uint8_t pad0;
  uint32_t pad1;
};
static_assert(sizeof(TcEntry) == 32, "TcEntry is 32 bytes");
// The tensor-core kernel reads task descriptors in chunks of kTcChunkCopy entries,
// kTcChunk apart: the entry array carries kTcChunkCopy zero entries after its end.
constexpr int kTcChunk = 56;
constexpr int kTcChunkCopy = 64;
struct TcGroup {
  uint64_t d;       // element offset of the output block (or scratch slot)
  int drs, dcs, m, q;
  int first, count;
};

// operator tiles from FP32 (src_f64 false) or FP64 sources (src == ~0: exact identity tile)
cudaError_t launch_build_tiles(const TileSpec *t, int ntiles, uint8_t *arena, bool src_f64, cudaStream_t s);
// Y^T tiles of FP64 psi blocks
cudaError_t launch_psi_tiles(const PsiTileSpec *t, int ntiles, const double *psi, uint8_t *arena,
                             cudaStream_t s);
// tensor-core H.psi chain (split-BF16 x3, FP32 accumulation, FP64 output blocks), persistent
// CTAs taking groups (m, q <= 128, every entry n, p <= 128) from *counter (zeroed here on s);
// shape 1: every group has m, q <= 64 and every entry p <= 64 (MMA M = 64, four CTAs per SM);
// shape 2: m <= 64, q and p <= 32 (five CTAs per SM); shape 0: the rest;
// *status (8 ints) is raised if an mbarrier wait ran out
// pipeline-wait limit of the tensor-core kernel (tries <= 0: the default)
void set_tc_wait_tries(long long tries);
cudaError_t launch_chain_tc2(const TcEntry *e, const TcGroup *g, int ngroups, const uint8_t *optiles,
                             const uint8_t *psitiles, uint64_t db, int *counter, int *status, int shape,
                             cudaStream_t s);

}  // namespace dmrg
