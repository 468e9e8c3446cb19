// tcgen05 (5th-generation tensor core) kernels for sm_103a.
//
// tc_selftest: one M=128 x N x K bf16 GEMM with FP32 accumulation in TMEM,
// used to validate the descriptor encodings on the device (C = A B^T).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "kernels.cuh"
#include "tc.cuh"

namespace dmrg {

static constexpr long long kMaxWaitTries = 1ll << 22;  // bounded mbarrier waits

// Polls of the tensor-core kernel's pipeline waits (the waits that order the
// jobs); the drain waits before TMEM is released and the CTA exits always take
// kMaxWaitTries.  Changed only by dmrg_debug_set_wait_limit, so that a test can
// make the pipeline waits run out and see the time-out reported: with 0 polls
// every pipeline wait gives up at once, before any copy or MMA is issued.
static std::atomic<long long> g_tc_wait_tries{kMaxWaitTries};

void set_tc_wait_tries(long long tries) { g_tc_wait_tries.store(tries >= 0 ? tries : kMaxWaitTries); }

__global__ void __launch_bounds__(128) tc_selftest_kernel(const float *__restrict__ A,
                                                          const float *__restrict__ B, float *C,
                                                          int N, int K, int *status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *As = smem;                 // 128 x 64 bf16, K-major core matrices (16 KB)
  uint8_t *Bs = smem + 16384;         // 256 x 64 bf16 (32 KB)
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 49152);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 49152 + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int KC = 64;
  if (warp == 0) {
    tc::tmem_alloc(tslot, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  for (int idx = tid; idx < 128 * KC; idx += 128) {
    const int r = idx / KC, k = idx % KC;
    const float a = (k < K) ? A[r * K + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16 *>(As + tc::kmajor_off(r, k, KC)) = __float2bfloat16_rn(a);
  }
  for (int idx = tid; idx < 256 * KC; idx += 128) {
    const int r = idx / KC, k = idx % KC;
    const float b = (r < N && k < K) ? B[r * K + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16 *>(Bs + tc::kmajor_off(r, k, KC)) = __float2bfloat16_rn(b);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, N);
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = tc::make_desc(tc::smem_u32(As) + ks * 2 * 128, 128, (KC / 8) * 128);
      const uint64_t bd = tc::make_desc(tc::smem_u32(Bs) + ks * 2 * 128, 128, (KC / 8) * 128);
      tc::mma_bf16(tbase, ad, bd, idesc, ks > 0 ? 1u : 0u);
    }
    tc::mma_commit(bar);
  }
  const bool ok = tc::mbar_wait(bar, 0, kMaxWaitTries);
  tc::fence_after();
  if (!ok) {
    if (tid == 0) atomicExch(status, 1);
  } else {
    const int row = tid;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) C[row * N + c0 + i] = v[i];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

cudaError_t launch_tc_selftest(const float *A, const float *B, float *C, int N, int K, int *status,
                               cudaStream_t s) {
  if (N < 16 || N > 256 || N % 16 || K < 16 || K > 64 || K % 16) return cudaErrorInvalidValue;
  const int smem = 49152 + 64;
  cudaError_t e = cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  tc_selftest_kernel<<<1, 128, smem, s>>>(A, B, C, N, K, status);
  return cudaGetLastError();
}

}  // namespace dmrg

namespace dmrg {

// ---------------------------------------------------------------------------
// Pre-split operand tiles and the pipelined tensor-core chain.
//
// Every operand the tensor core reads from global memory is stored once as a
// ready-made shared-memory image: rows padded to R16 = ceil16(R) and K to
// K16 = ceil16(K) with zeros, cut into K chunks of T2_W columns (the last one
// narrower when T2_W does not divide K16).  Chunk c starts at byte
// 4 * T2_W * R16 * c and holds the bf16 hi part (R16 x w, K-major core
// matrices, core matrix (rg, kg) at (rg * w/8 + kg) * 128) followed by the lo
// part.  A chunk is one 1-D bulk copy (cp.async.bulk) into shared memory, so
// staging costs no thread work.
//
// Operator blocks (X and Z^T views of the stored and pre-summed operators)
// are tiled once per task list; the psi blocks (as Y^T) once per H.psi call.
// ---------------------------------------------------------------------------

static constexpr int T2_W = 32;  // K chunk width (elements); a chunk of R16 rows is 4 * T2_W * R16 bytes

template <typename Load>
__device__ __forceinline__ void write_tile(uint8_t *img, int R, int K, Load load, int t0, int nt) {
  const int R16 = (R + 15) & ~15, K16 = (K + 15) & ~15;
  const int units = R16 * (K16 >> 3);
  for (int u = t0; u < units; u += nt) {
    const int r = u % R16, kg = u / R16, k0 = kg * 8;
    const int c = k0 / T2_W, w = min(T2_W, K16 - c * T2_W), kgi = (k0 - c * T2_W) >> 3;
    uint8_t *hi = img + (size_t)4 * T2_W * R16 * c + ((r >> 3) * (w >> 3) + kgi) * 128 + (r & 7) * 16;
    uint8_t *lo = hi + (size_t)R16 * w * 2;
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float x = (r < R && k0 + i < K) ? load(r, k0 + i) : 0.f;
      tc::split_bf16(x, h[i], l[i]);
    }
    *reinterpret_cast<uint4 *>(hi) = *reinterpret_cast<const uint4 *>(h);
    *reinterpret_cast<uint4 *>(lo) = *reinterpret_cast<const uint4 *>(l);
  }
}

// Tiles of operator views; the sources are FP32 copies or the FP64 masters (SRC).
template <typename SRC>
__global__ void __launch_bounds__(256) build_tiles_kernel(const TileSpec *__restrict__ T, int ntiles,
                                                          uint8_t *arena) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileSpec s = T[t];
    uint8_t *img = arena + s.dst;
    if (s.src == ~0ull) {
      write_tile(img, s.R, s.K, [](int r, int k) { return r == k ? 1.f : 0.f; }, threadIdx.x, blockDim.x);
    } else {
      const SRC *X = reinterpret_cast<const SRC *>(s.src);
      const int64_t rs = s.rs, cs = s.cs;
      write_tile(img, s.R, s.K, [&](int r, int k) { return (float)X[r * rs + k * cs]; }, threadIdx.x,
                 blockDim.x);
    }
  }
}

// Y^T of a psi block: tile row j (< p), column k (< n) is psi[src + k * p + j].
__global__ void __launch_bounds__(256) psi_tiles_kernel(const PsiTileSpec *__restrict__ T, int ntiles,
                                                        const double *__restrict__ psi, uint8_t *arena) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const PsiTileSpec s = T[t];
    const double *Y = psi + s.src;
    const int p = s.p;
    write_tile(arena + s.dst, s.p, s.n, [&](int j, int k) { return (float)Y[(int64_t)k * p + j]; },
               threadIdx.x, blockDim.x);
  }
}

cudaError_t launch_build_tiles(const TileSpec *t, int ntiles, uint8_t *arena, bool src_f64, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  add_kernel_launches(1);
  if (src_f64)
    build_tiles_kernel<double><<<std::min(ntiles, 152 * 16), 256, 0, s>>>(t, ntiles, arena);
  else
    build_tiles_kernel<float><<<std::min(ntiles, 152 * 16), 256, 0, s>>>(t, ntiles, arena);
  return cudaGetLastError();
}

cudaError_t launch_psi_tiles(const PsiTileSpec *t, int ntiles, const double *psi, uint8_t *arena,
                             cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  add_kernel_launches(1);
  psi_tiles_kernel<<<std::min(ntiles, 152 * 16), 256, 0, s>>>(t, ntiles, psi, arena);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// chain_tc2: D += sum_e f_e X_e Y_e Z_e per output block on the tensor cores
// (split-BF16 three-pass products, FP32 accumulation in TMEM).  Persistent:
// CTAS CTAs per SM, with TMEM, mbarriers and the zeroed stage ring set up once
// per CTA; the producer takes the next output block from a global counter
// (dynamic balance: a block's cost on the tensor cores is not its FLOP count)
// and hands the indices to the other roles through a small ring (gfull /
// gempty mbarriers; -1 ends the work).
//
// The tasks of an output block come in stacks: consecutive tasks that read the
// same psi block Y (TcEntry::stack on the first).  The work of a stack is a
// sequence of "jobs", one per K chunk:
//   stage 1 (K = n):  [T_1; T_2; ..] = [X_1; X_2; ..] Y
//                     A = the members' X chunks stacked along M, B = Y^T chunk
//   stage 2 (K = p), for each member i:  D += (f_i T_i) Z_i
//                     A = f_i T_i chunk written by the converter warps from
//                     TMEM (rows of member i), B = Z_i^T chunk
// Operand chunks are bulk-copied; identity X / Z are exact identity tiles.
// Jobs run through a ring of T2_NS shared-memory stages (A half, MR rows, |
// B half, TC rows; T2_W columns hi + lo) with warp roles:
//   warps 0-3  converters: T (TMEM lanes = rows) -> f T split into bf16 hi/lo
//              in stage 2 jobs; at the end of a block D (TMEM) -> FP64 output
//   warp 4     producer: bulk copies of the operand chunks
//   warp 5     MMA issuer: one thread issues tcgen05.mma and commits
// mbarriers per stage: full (copies landed), cvf (converters wrote A),
// empty (MMAs that read the stage finished); per stack: tfull (T complete),
// tempty (converters finished reading T); per output block: dfull (D
// complete), dempty (converters finished reading D).  Phases run on across
// stacks and blocks; every role derives the same job sequence.
// Every wait is bounded: on time-out the CTA raises *status, all roles stop,
// copies and MMAs in flight are waited for, and TMEM is released.
// ---------------------------------------------------------------------------

static constexpr int T2_NS = 3;
static constexpr int T2_MAXSTACK = 8;  // tasks stacked along M in one stage 1 (128 rows / 16)
// Task descriptors reach the roles through a ring of T2_DR shared-memory chunks,
// each one bulk copy of T2_DCOPY entries: the stacks that start among the
// chunk's first T2_DC entries (a stack has at most T2_MAXSTACK members, so all of
// them are in the copy).  The producer requests chunks ahead of use, so no role
// waits on a global load per stack.
static constexpr int T2_DR = 3;
static constexpr int T2_DC = kTcChunk;
static constexpr int T2_DCOPY = kTcChunkCopy;
static_assert(T2_DCOPY >= T2_DC + T2_MAXSTACK, "a chunk copy holds every stack that starts in it");
static constexpr int T2_THREADS = 192;

// Three shapes of the kernel, by the size of the output blocks they take:
//   T2Shape<128, 128, 2>: MMA M = 128, T and D 128 TMEM columns each, two CTAs per SM
//   T2Shape< 64,  64, 4>: m <= 64, q and every task's p <= 64, four CTAs per SM
//   T2Shape< 64,  32, 5>: m <= 64, q and every task's p <= 32, five CTAs per SM
// More resident CTAs hide more of the per-task latency of small blocks.  With
// M = 64 the accumulator row r sits in TMEM lane 32 (r / 16) + r % 16.
template <int MR, int TC, int CTAS>
struct T2Shape {
  static constexpr int AHALF = MR * T2_W * 4;  // A operand of a stage: MR rows, hi + lo
  static constexpr int BHALF = TC * T2_W * 4;  // B operand: at most TC rows, hi + lo
  static constexpr int ALO = MR * T2_W * 2;    // lo part of the converter-written A operand
  static constexpr int STAGE = AHALF + BHALF;
  static constexpr int DESC_OFF = T2_NS * STAGE;  // ring of task-descriptor chunks
  static constexpr int BAR_OFF = DESC_OFF + T2_DR * T2_DCOPY * (int)sizeof(TcEntry);
  static constexpr int TCOLS = TC;             // T and D regions of TMEM
  static constexpr int CTAS_PER_SM = CTAS;
  static constexpr int SMEM_LAUNCH = CTAS == 2 ? 104 * 1024 : CTAS == 4 ? 55 * 1024 : 44 * 1024;
  // accumulator row held by TMEM lane L (-1: none)
  __device__ static __forceinline__ int row_of_lane(int L) {
    if (MR == 128) return L;
    return (L & 31) < 16 ? (L >> 5) * 16 + (L & 31) : -1;
  }
};

static constexpr int T2_GR = 4;  // ring of fetched output-block indices

struct T2Bars {
  uint64_t full[T2_NS], cvf[T2_NS], empty[T2_NS];
  uint64_t tfull, tempty, dfull, dempty, drain;
  uint64_t gfull[T2_GR], gempty[T2_GR];
  uint64_t qfull[T2_DR], qempty[T2_DR];  // descriptor chunks: landed / released by all six roles
  TcGroup gdesc[T2_GR];                  // header of each published output block
  int gidx[T2_GR];
  uint32_t tslot;
  int abort;
};

// Time-out record: status[0] = 1; the first CTA to time out also fills
// status[1..7] = wait site, parity, block, aux0, aux1, raw mbarrier word (lo, hi)
__device__ __noinline__ void t2_timeout(int *status, uint64_t *bar, int site, uint32_t parity, int aux0,
                                        int aux1) {
  atomicExch(status, 1);
  if (atomicCAS(status + 1, 0, site) == 0) {
    const unsigned long long w = *reinterpret_cast<volatile unsigned long long *>(bar);
    status[2] = (int)parity;
    status[3] = (int)blockIdx.x;
    status[4] = aux0;
    status[5] = aux1;
    status[6] = (int)(w & 0xffffffffu);
    status[7] = (int)(w >> 32);
  }
}

// single-thread bounded wait that gives up early when another role aborted
__device__ __forceinline__ bool t2_wait1(uint64_t *bar, uint32_t parity, volatile int *abort, int *status,
                                         int site, int aux0, int aux1, long long tries) {
  for (long long i = 0; i < tries; ++i) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && *abort) return false;
  }
  *abort = 1;
  t2_timeout(status, bar, site, parity, aux0, aux1);
  return false;
}

// warp-uniform bounded wait (all 32 lanes take the same decision)
__device__ __forceinline__ bool t2_waitw(uint64_t *bar, uint32_t parity, volatile int *abort, int *status,
                                         int site, int aux0, int aux1, long long tries) {
  for (long long i = 0; i < tries; ++i) {
    if (__all_sync(0xffffffffu, tc::mbar_try_wait(bar, parity))) return true;
    if ((i & 63) == 63 && __any_sync(0xffffffffu, *abort)) return false;
  }
  if ((threadIdx.x & 31) == 0) {
    *abort = 1;
    t2_timeout(status, bar, site, parity, aux0, aux1);
  }
  __syncwarp();
  return false;
}

__device__ __forceinline__ int ceil16(int x) { return (x + 15) & ~15; }

// Stage-2 jobs: when the inner dimension p of a stack is at most 16, the K chunk
// is 16 wide and two members share one job (their A tiles side by side in the
// stage's A half, their Z^T tiles side by side in its B half, one MMA chain
// each into D); otherwise one member per job.
__device__ __forceinline__ int t2_members_per_job(int p16) { return p16 == 16 ? 2 : 1; }

template <int MR, int TC, int CTAS>
__global__ void __launch_bounds__(T2_THREADS, CTAS) chain_tc2_kernel(const TcEntry *__restrict__ E,
                                                               const TcGroup *__restrict__ G, int ngroups,
                                                               const uint8_t *__restrict__ optiles,
                                                               const uint8_t *__restrict__ psitiles,
                                                               uint64_t db, int *counter, int *status,
                                                               long long tries) {
  extern __shared__ __align__(1024) uint8_t smem[];
  using S = T2Shape<MR, TC, CTAS>;
  T2Bars *B = reinterpret_cast<T2Bars *>(smem + S::BAR_OFF);
  TcEntry *dring = reinterpret_cast<TcEntry *>(smem + S::DESC_OFF);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&B->tslot, 2 * S::TCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < T2_NS; ++s) {
      tc::mbar_init(&B->full[s], 1);
      tc::mbar_init(&B->cvf[s], 4);
      tc::mbar_init(&B->empty[s], 1);
    }
    tc::mbar_init(&B->tfull, 1);
    tc::mbar_init(&B->tempty, 4);
    tc::mbar_init(&B->dfull, 1);
    tc::mbar_init(&B->dempty, 4);
    tc::mbar_init(&B->drain, 1);
    for (int r = 0; r < T2_GR; ++r) {
      tc::mbar_init(&B->gfull[r], 1);
      tc::mbar_init(&B->gempty[r], 5);  // MMA issuer + 4 converter warps
    }
    for (int s = 0; s < T2_DR; ++s) {
      tc::mbar_init(&B->qfull[s], 1);
      tc::mbar_init(&B->qempty[s], 6);  // producer + MMA issuer + 4 converter warps
    }
    B->abort = 0;
  }
  // A halves: rows beyond a block's 16-row padding only feed discarded TMEM lanes,
  // but must hold finite values (B halves are read only where copied)
  for (int i = tid; i < T2_NS * (S::AHALF / 16); i += T2_THREADS) {
    const int s = i / (S::AHALF / 16), o = i % (S::AHALF / 16);
    reinterpret_cast<uint4 *>(smem + s * S::STAGE)[o] = make_uint4(0, 0, 0, 0);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = B->tslot, tT = tbase, tD = tbase + S::TCOLS;
  volatile int *abort = &B->abort;
  volatile int *gidx = B->gidx;
  // descriptor chunk q (the CTA's running chunk count) lives in ring slot q % T2_DR
  auto chunk = [&](int q) { return dring + (q % T2_DR) * T2_DCOPY; };

  if (warp == 4) {
    // ---------------- producer
    if (lane == 0) {
      int j = 0, qacc = 0, qreq = 0;
      int qlast[T2_DR];
#pragma unroll
      for (int s = 0; s < T2_DR; ++s) qlast[s] = -1;
      bool ok = true;
      for (int gl = 0; ok; ++gl) {
        // take the next output block and publish it (index and header) to the other roles
        const int r = gl % T2_GR;
        if (!t2_wait1(&B->gempty[r], ((uint32_t)(gl / T2_GR) & 1u) ^ 1u, abort, status, 101, j, gl, tries)) break;
        const int gi0 = atomicAdd(counter, 1);
        const int gi = gi0 < ngroups ? gi0 : -1;
        TcGroup g{};
        if (gi >= 0) g = G[gi];
        B->gdesc[r] = g;
        gidx[r] = gi;
        tc::mbar_arrive(&B->gfull[r]);  // release: index and header are visible to the waiters
        if (gi < 0) break;
        const int m16 = ceil16(g.m), q16 = ceil16(g.q), e_end = g.first + g.count;
        const int nch = (g.count + T2_DC - 1) / T2_DC;
        // request descriptor chunks up to T2_DR - 1 ahead of the one in use
        auto request_upto = [&](int qhi) {
          for (; ok && qreq <= qhi && qreq < qacc + nch; ++qreq) {
            const int s = qreq % T2_DR;
            const uint32_t u = (uint32_t)(qreq / T2_DR);
            if (!t2_wait1(&B->qempty[s], (u & 1u) ^ 1u, abort, status, 114, j, qreq, tries)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&B->qfull[s], T2_DCOPY * (uint32_t)sizeof(TcEntry));
            tc::bulk_g2s(chunk(qreq), E + g.first + (size_t)(qreq - qacc) * T2_DC,
                         T2_DCOPY * (uint32_t)sizeof(TcEntry), &B->qfull[s]);
            qlast[s] = qreq;
          }
        };
        int ei = g.first;
        for (int c = 0; c < nch && ok; ++c) {
          const int q = qacc + c;
          request_upto(q + T2_DR - 1);
          if (!ok || !t2_wait1(&B->qfull[q % T2_DR], (uint32_t)(q / T2_DR) & 1u, abort, status, 115, j, q,
                               tries)) {
            ok = false;
            break;
          }
          const TcEntry *D0 = chunk(q);  // entry e of this block at D0[e - e0]
          const int e0 = g.first + c * T2_DC;
          const int c_end = min(e_end, g.first + (c + 1) * T2_DC);
          for (; ei < c_end && ok;) {
            const int ns = min(max((int)D0[ei - e0].stack, 1), T2_MAXSTACK);
            const int n16 = ceil16(D0[ei - e0].n), p16 = ceil16(D0[ei - e0].p);
            const uint32_t yt = D0[ei - e0].yt;
            const int nch1 = (n16 + T2_W - 1) / T2_W, nch2 = (p16 + T2_W - 1) / T2_W;
            // stage 1 of the stack: the X chunks of every member, rows stacked, and one Y^T chunk
            for (int cc = 0; cc < nch1 && ok; ++cc, ++j) {
              const int s = j % T2_NS;
              const uint32_t u = (uint32_t)(j / T2_NS);
              if (!t2_wait1(&B->empty[s], (u & 1u) ^ 1u, abort, status, 102, j, (int)u, tries)) {
                ok = false;
                break;
              }
              uint8_t *st = smem + s * S::STAGE;
              const int w = min(T2_W, n16 - cc * T2_W);
              const uint32_t bx = (uint32_t)(m16 * w * 2), by = (uint32_t)(p16 * w * 4);
              tc::mbar_arrive_expect_tx(&B->full[s], 2 * bx * ns + by);
              for (int i = 0; i < ns; ++i) {
                const uint8_t *src = optiles + D0[ei - e0 + i].xt + (uint64_t)4 * T2_W * m16 * cc;
                tc::bulk_g2s(st + i * bx, src, bx, &B->full[s]);                 // hi rows
                tc::bulk_g2s(st + S::ALO + i * bx, src + bx, bx, &B->full[s]);   // lo rows
              }
              tc::bulk_g2s(st + S::AHALF, psitiles + yt + (uint64_t)4 * T2_W * p16 * cc, by, &B->full[s]);
            }
            // stage 2: the members' Z^T chunks (two members to a job when K is 16 wide)
            const int per = t2_members_per_job(p16);
            for (int i0 = 0; i0 < ns && ok; i0 += per) {
              const int nm = min(per, ns - i0);
              for (int cc = 0; cc < nch2 && ok; ++cc, ++j) {
                const int s = j % T2_NS;
                const uint32_t u = (uint32_t)(j / T2_NS);
                if (!t2_wait1(&B->empty[s], (u & 1u) ^ 1u, abort, status, 103, j, (int)u, tries)) {
                  ok = false;
                  break;
                }
                const int w = min(T2_W, p16 - cc * T2_W);
                const uint32_t bz = (uint32_t)(q16 * w * 4);
                tc::mbar_arrive_expect_tx(&B->full[s], bz * nm);
                for (int t = 0; t < nm; ++t)
                  tc::bulk_g2s(smem + s * S::STAGE + S::AHALF + t * bz,
                               optiles + D0[ei - e0 + i0 + t].zt + (uint64_t)4 * T2_W * q16 * cc, bz, &B->full[s]);
              }
            }
            ei += ns;
          }
          if (ok) tc::mbar_arrive(&B->qempty[q % T2_DR]);  // done with this chunk's descriptors
        }
        qacc += nch;
      }
      // copies in flight land before the CTA exits (bounded)
      for (int s = 0; s < T2_NS; ++s) {
        int jl = j - 1;
        while (jl >= 0 && jl % T2_NS != s) --jl;
        if (jl >= 0) tc::mbar_wait(&B->full[s], (uint32_t)(jl / T2_NS) & 1u, kMaxWaitTries);
      }
      for (int s = 0; s < T2_DR; ++s)
        if (qlast[s] >= 0) tc::mbar_wait(&B->qfull[s], (uint32_t)(qlast[s] / T2_DR) & 1u, kMaxWaitTries);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int j = 0, ls = 0, gl = 0, qacc = 0;
      uint32_t cvpar = 0;
      bool ok = true;
      for (; ok; ++gl) {
        const int r = gl % T2_GR;
        if (!t2_wait1(&B->gfull[r], (uint32_t)(gl / T2_GR) & 1u, abort, status, 104, j, ls, tries)) break;
        const int gi = gidx[r];
        const TcGroup g = B->gdesc[r];
        tc::mbar_arrive(&B->gempty[r]);
        if (gi < 0) break;
        const int q16 = ceil16(g.q), e_end = g.first + g.count;
        const int nch = (g.count + T2_DC - 1) / T2_DC;
        const uint32_t id2 = tc::idesc_bf16(MR, q16);
        bool dfirst = true;
        int ei = g.first;
        for (int c = 0; c < nch && ok; ++c) {
          const int q = qacc + c;
          if (!t2_wait1(&B->qfull[q % T2_DR], (uint32_t)(q / T2_DR) & 1u, abort, status, 116, j, q, tries)) {
            ok = false;
            break;
          }
          const TcEntry *D0 = chunk(q);
          const int e0 = g.first + c * T2_DC;
          const int c_end = min(e_end, g.first + (c + 1) * T2_DC);
          for (; ei < c_end && ok; ++ls) {
            const int ns = min(max((int)D0[ei - e0].stack, 1), T2_MAXSTACK);
            const int n16 = ceil16(D0[ei - e0].n), p16 = ceil16(D0[ei - e0].p);
            const int nch1 = (n16 + T2_W - 1) / T2_W, nch2 = (p16 + T2_W - 1) / T2_W;
            if (ls > 0) {  // T of the previous stack has been read
              if (!t2_wait1(&B->tempty, (uint32_t)(ls - 1) & 1u, abort, status, 105, j, ls, tries)) {
                ok = false;
                break;
              }
              tc::fence_after();
            }
            const uint32_t id1 = tc::idesc_bf16(MR, p16);
            for (int cc = 0; cc < nch1 && ok; ++cc, ++j) {
              const int s = j % T2_NS;
              const uint32_t u = (uint32_t)(j / T2_NS);
              if (!t2_wait1(&B->full[s], u & 1u, abort, status, 106, j, ls, tries)) {
                ok = false;
                break;
              }
              tc::fence_after();
              const int w = min(T2_W, n16 - cc * T2_W);
              const uint32_t sbo = (uint32_t)(w / 8) * 128;
              const uint32_t a = tc::smem_u32(smem + s * S::STAGE), b = a + S::AHALF;
              const uint32_t alo = a + S::ALO, blo = b + (uint32_t)(p16 * w * 2);
              for (int ks = 0; ks < w / 16; ++ks) {
                const uint32_t o = (uint32_t)ks * 256;
                tc::mma_bf16(tT, tc::make_desc(a + o, 128, sbo), tc::make_desc(b + o, 128, sbo), id1,
                             (cc == 0 && ks == 0) ? 0u : 1u);
                tc::mma_bf16(tT, tc::make_desc(a + o, 128, sbo), tc::make_desc(blo + o, 128, sbo), id1, 1u);
                tc::mma_bf16(tT, tc::make_desc(alo + o, 128, sbo), tc::make_desc(b + o, 128, sbo), id1, 1u);
              }
              tc::mma_commit(&B->empty[s]);
            }
            if (!ok) break;
            tc::mma_commit(&B->tfull);
            if (dfirst && gl > 0) {  // D of the previous block has been written out
              if (!t2_wait1(&B->dempty, (uint32_t)(gl - 1) & 1u, abort, status, 107, j, ls, tries)) {
                ok = false;
                break;
              }
              tc::fence_after();
            }
            const int per = t2_members_per_job(p16);
            for (int i0 = 0; i0 < ns && ok; i0 += per) {
              const int nm = min(per, ns - i0);
              for (int cc = 0; cc < nch2 && ok; ++cc, ++j) {
                const int s = j % T2_NS;
                const uint32_t u = (uint32_t)(j / T2_NS);
                if (!t2_wait1(&B->full[s], u & 1u, abort, status, 108, j, ls, tries) ||
                    !t2_wait1(&B->cvf[s], (cvpar >> s) & 1u, abort, status, 109, j, ls, tries)) {
                  ok = false;
                  break;
                }
                cvpar ^= 1u << s;
                tc::fence_after();
                const int w = min(T2_W, p16 - cc * T2_W);
                const uint32_t sbo = (uint32_t)(w / 8) * 128;
                const uint32_t a0 = tc::smem_u32(smem + s * S::STAGE);
                for (int t = 0; t < nm; ++t) {  // member t of the job: its A tile and its B tile
                  const uint32_t a = a0 + (uint32_t)(t * MR * w * 2), alo = a + S::ALO;
                  const uint32_t b = a0 + S::AHALF + (uint32_t)(t * q16 * w * 4), blo = b + (uint32_t)(q16 * w * 2);
                  for (int ks = 0; ks < w / 16; ++ks) {
                    const uint32_t o = (uint32_t)ks * 256;
                    tc::mma_bf16(tD, tc::make_desc(a + o, 128, sbo), tc::make_desc(b + o, 128, sbo), id2,
                                 dfirst ? 0u : 1u);
                    dfirst = false;
                    tc::mma_bf16(tD, tc::make_desc(a + o, 128, sbo), tc::make_desc(blo + o, 128, sbo), id2, 1u);
                    tc::mma_bf16(tD, tc::make_desc(alo + o, 128, sbo), tc::make_desc(b + o, 128, sbo), id2, 1u);
                  }
                }
                tc::mma_commit(&B->empty[s]);
              }
            }
            ei += ns;
          }
          if (ok) tc::mbar_arrive(&B->qempty[q % T2_DR]);
        }
        qacc += nch;
        if (ok) tc::mma_commit(&B->dfull);
      }
      tc::mma_commit(&B->drain);  // every MMA issued above has finished before TMEM is released
      tc::mbar_wait(&B->drain, 0, kMaxWaitTries);
    }
  } else {
    // ---------------- converters (thread = TMEM lane = accumulator row, if any)
    const int R = S::row_of_lane(tid);
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    int j = 0, ls = 0, gl = 0, qacc = 0;
    bool ok = true;
    for (; ok; ++gl) {
      const int r = gl % T2_GR;
      if (!t2_waitw(&B->gfull[r], (uint32_t)(gl / T2_GR) & 1u, abort, status, 110, j, ls, tries)) break;
      const int gi = gidx[r];
      const TcGroup g = B->gdesc[r];
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&B->gempty[r]);
      if (gi < 0) break;
      const int m = g.m, q = g.q, m16 = ceil16(m), q16 = ceil16(q), e_end = g.first + g.count;
      const int nch = (g.count + T2_DC - 1) / T2_DC;
      // this thread's T row belongs to stack member R / m16, output row R % m16
      const int mine = R >= 0 ? R / m16 : -1, orow = R >= 0 ? R % m16 : 0;
      int ei = g.first;
      for (int c = 0; c < nch && ok; ++c) {
        const int qc = qacc + c;
        if (!t2_waitw(&B->qfull[qc % T2_DR], (uint32_t)(qc / T2_DR) & 1u, abort, status, 117, j, qc, tries)) {
          ok = false;
          break;
        }
        const TcEntry *D0 = chunk(qc);
        const int e0 = g.first + c * T2_DC;
        const int c_end = min(e_end, g.first + (c + 1) * T2_DC);
        for (; ei < c_end && ok; ++ls) {
          const int ns = min(max((int)D0[ei - e0].stack, 1), T2_MAXSTACK);
          const int n16 = ceil16(D0[ei - e0].n), p16 = ceil16(D0[ei - e0].p);
          const int nch1 = (n16 + T2_W - 1) / T2_W, nch2 = (p16 + T2_W - 1) / T2_W;
          const float f = mine >= 0 && mine < ns ? D0[ei - e0 + mine].f : 0.f;
          j += nch1;
          if (!t2_waitw(&B->tfull, (uint32_t)ls & 1u, abort, status, 111, j, ls, tries)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const int per = t2_members_per_job(p16);
          for (int i0 = 0; i0 < ns && ok; i0 += per) {
            const int nm = min(per, ns - i0);
            const bool writes = mine >= i0 && mine < i0 + nm && orow < m;
            const int t = writes ? mine - i0 : 0;  // this thread's member within the job
            // a warp that holds no T row of this job's members only signals (the
            // TMEM load is warp-collective, so the test is warp-uniform)
            const int r_lo = i0 * m16, r_hi = (i0 + nm - 1) * m16 + m;
            const int w_lo = (MR == 128 ? 32 : 16) * warp, w_hi = w_lo + (MR == 128 ? 32 : 16);
            const bool warp_busy = r_lo < w_hi && w_lo < r_hi;
            for (int cc = 0; cc < nch2; ++cc, ++j) {
              const int s = j % T2_NS;
              const uint32_t u = (uint32_t)(j / T2_NS);
              if (!t2_waitw(&B->empty[s], (u & 1u) ^ 1u, abort, status, 112, j, (int)u, tries)) {
                ok = false;
                break;
              }
              tc::fence_after();
              const int w = min(T2_W, p16 - cc * T2_W);
              uint8_t *A = smem + s * S::STAGE + t * MR * w * 2;
              if (warp_busy) {
                float v[2][16];
                const uint32_t ta = tT + lane_off + (uint32_t)(cc * T2_W);
                if (w == 32) {
                  tc::tmem_ld16x2(ta, ta + 16, v[0], v[1]);
                } else {
                  tc::tmem_ld16(ta, v[0]);
                }
                if (writes) {
#pragma unroll
                  for (int h = 0; h < 2; ++h) {
                    if (h * 16 >= w) break;
#pragma unroll
                    for (int g2 = 0; g2 < 2; ++g2) {
                      __align__(16) __nv_bfloat16 hb[8], lb[8];
#pragma unroll
                      for (int k = 0; k < 8; ++k) tc::split_bf16(f * v[h][8 * g2 + k], hb[k], lb[k]);
                      uint8_t *dst = A + ((orow >> 3) * (w >> 3) + 2 * h + g2) * 128 + (orow & 7) * 16;
                      *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(hb);
                      *reinterpret_cast<uint4 *>(dst + S::ALO) = *reinterpret_cast<const uint4 *>(lb);
                    }
                  }
                }
              }
              tc::fence_async_smem();
              __syncwarp();
              if (lane == 0) tc::mbar_arrive(&B->cvf[s]);
            }
          }
          if (!ok) break;
          tc::fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&B->tempty);
          ei += ns;
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&B->qempty[qc % T2_DR]);
      }
      qacc += nch;
      if (!ok) break;
      // ---- output block: D (TMEM) -> FP64 global, then release D
      if (!t2_waitw(&B->dfull, (uint32_t)gl & 1u, abort, status, 113, j, ls, tries)) {
        ok = false;
        break;
      }
      tc::fence_after();
      double *Dout = reinterpret_cast<double *>(db + g.d * 8ull);
      for (int c0 = 0; c0 < q16; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tD + lane_off + (uint32_t)c0, v);
        if (R >= 0 && R < m) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < q) Dout[(int64_t)R * g.drs + (int64_t)(c0 + i) * g.dcs] += (double)v[i];
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&B->dempty);
    }
  }
  __syncwarp();  // lanes 1-31 of the producer and MMA warps rejoin lane 0
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 2 * S::TCOLS);
}

template <int MR, int TC, int CTAS>
static cudaError_t launch_tc2_shape(const TcEntry *e, const TcGroup *g, int ngroups, const uint8_t *optiles,
                                   const uint8_t *psitiles, uint64_t db, int *counter, int *status,
                                   cudaStream_t s) {
  const long long tries = g_tc_wait_tries.load();
  using S = T2Shape<MR, TC, CTAS>;
  static_assert(S::BAR_OFF + (int)sizeof(T2Bars) <= S::SMEM_LAUNCH, "shared memory budget");
  // the launch size caps resident CTAs per SM at CTAS, so their TMEM fits the SM's 512 columns
  static_assert((CTAS + 1) * (S::SMEM_LAUNCH + 1024) > 228 * 1024, "more resident CTAs than intended");
  static_assert(CTAS * 2 * TC <= 512, "TMEM oversubscription");
  cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (err != cudaSuccess) return err;
  auto kern = chain_tc2_kernel<MR, TC, CTAS>;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM_LAUNCH);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  const int grid = std::min(ngroups, CTAS * std::max(sms, 1));
  add_kernel_launches(1);
  kern<<<grid, T2_THREADS, S::SMEM_LAUNCH, s>>>(e, g, ngroups, optiles, psitiles, db, counter, status, tries);
  return cudaGetLastError();
}

cudaError_t launch_chain_tc2(const TcEntry *e, const TcGroup *g, int ngroups, const uint8_t *optiles,
                             const uint8_t *psitiles, uint64_t db, int *counter, int *status, int shape,
                             cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  if (shape == 2) return launch_tc2_shape<64, 32, 5>(e, g, ngroups, optiles, psitiles, db, counter, status, s);
  if (shape == 1) return launch_tc2_shape<64, 64, 4>(e, g, ngroups, optiles, psitiles, db, counter, status, s);
  return launch_tc2_shape<128, 128, 2>(e, g, ngroups, optiles, psitiles, db, counter, status, s);
}

}  // namespace dmrg
