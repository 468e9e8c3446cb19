// FP64 device kernels of the two-site QC-DMRG hot path (sm_103a).
//
// chain_fp64:   batched triple product D += sum_e f_e X_e Y_e Z_e over a task
//               list grouped by output block (one CTA owns each 32x32 output
//               tile, so accumulation is deterministic and needs no atomics).
//               Used for H.psi (Sec. 2.2.1, Eq. dgemm: X = A_l, Y = psi^s,
//               Z = A_r^T), for the renormalization O^T (A (x) o) O of
//               Sec. 2.2.2 / Eq. renorm_mat (X = O^T, Y = A, Z = O) and for
//               the density matrix psi psi^T of Sec. 2.1.
// lincomb_fp64: pre-summed operators (Sec. 2.2.3, Eq. presum) as a GEMM
//               [K_out x K_src] x [K_src x block elements] per sector.
// Davidson helpers, a round-robin parallel Jacobi eigensolver for the small subspace
// matrix, and a column gather that builds O from eigenvectors.
#include <cuda_runtime.h>

#include <atomic>

#include "kernels.cuh"

namespace dmrg {

#define IDN (~0ull)

static std::atomic<long long> g_launches{0};
long long kernel_launch_count() { return g_launches.load(); }
void add_kernel_launches(long long n) { g_launches.fetch_add(n); }
#define COUNT(n) g_launches.fetch_add(n)

__device__ __forceinline__ const double *dptr(uint64_t base, uint64_t off) {
  return reinterpret_cast<const double *>(base + off * 8ull);
}

template <typename T>
__device__ __forceinline__ const T *tptr(uint64_t base, uint64_t off) {
  return reinterpret_cast<const T *>(base + off * sizeof(T));
}

// TX/TY/TZ: operand element types; TA: accumulation type; D is FP64.
template <typename TX, typename TY, typename TZ, typename TA>
__global__ void __launch_bounds__(256) chain_kernel(const ChainEntry *__restrict__ E,
                                                    const ChainGroup *__restrict__ G, int ngroups,
                                                    uint64_t xb, uint64_t yb, uint64_t zb,
                                                    uint64_t db) {
  __shared__ TA Xs[32][33];
  __shared__ TA Ys[32][33];
  __shared__ TA Ts[32][33];
  __shared__ TA Zs[32][33];
  const int tile = blockIdx.x;
  int lo = 0, hi = ngroups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (G[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  const ChainGroup g = G[lo];
  const int ntq = (g.q + 31) >> 5;
  const int tl = tile - g.tile0;
  const int r0 = (tl / ntq) * 32, c0 = (tl % ntq) * 32;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int mrows = min(32, g.m - r0), qcols = min(32, g.q - c0);
  TA acc[4] = {0, 0, 0, 0};

  for (int ei = g.first; ei < g.first + g.count; ++ei) {
    const ChainEntry e = E[ei];
    const bool xid = e.x == IDN, yid = e.y == IDN, zid = e.z == IDN;
    const TX *X = xid ? nullptr : tptr<TX>(xb, e.x);
    const TY *Y = yid ? nullptr : tptr<TY>(yb, e.y);
    const TZ *Z = zid ? nullptr : tptr<TZ>(zb, e.z);
    const TA f = (TA)e.f;
    const int n = e.n, p = e.p;
    const int pbeg = zid ? c0 : 0;
    const int pend = zid ? min(c0 + 32, p) : p;
    for (int p0 = pbeg; p0 < pend; p0 += 32) {
      const int pc = min(32, pend - p0);
      TA t[4] = {0, 0, 0, 0};
      if (xid || yid) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = ty + 8 * i;
          if (r < mrows && tx < pc) {
            const int64_t R = r0 + r, Cc = p0 + tx;
            if (xid && yid) t[i] = (R == Cc) ? (TA)1 : (TA)0;
            else if (xid) t[i] = (TA)Y[R * e.yrs + Cc * e.ycs];
            else t[i] = (TA)X[R * e.xrs + Cc * e.xcs];
          }
        }
      } else {
        for (int n0 = 0; n0 < n; n0 += 32) {
          const int nc = min(32, n - n0);
          for (int idx = tid; idx < 1024; idx += 256) {
            const int i = idx >> 5, kk = idx & 31;
            Xs[i][kk] = (i < mrows && kk < nc)
                            ? (TA)X[(int64_t)(r0 + i) * e.xrs + (int64_t)(n0 + kk) * e.xcs] : (TA)0;
            Ys[i][kk] = (i < nc && kk < pc)
                            ? (TA)Y[(int64_t)(n0 + i) * e.yrs + (int64_t)(p0 + kk) * e.ycs] : (TA)0;
          }
          __syncthreads();
          if (tx < pc) {
            for (int kk = 0; kk < nc; ++kk) {
              const TA y = Ys[kk][tx];
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (ty + 8 * i < mrows) t[i] = fma(Xs[ty + 8 * i][kk], y, t[i]);
            }
          }
          __syncthreads();
        }
      }
      if (zid) {
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = fma(f, t[i], acc[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) Ts[ty + 8 * i][tx] = t[i];
        for (int idx = tid; idx < 1024; idx += 256) {
          const int kk = idx >> 5, j = idx & 31;
          Zs[kk][j] = (kk < pc && j < qcols)
                          ? (TA)Z[(int64_t)(p0 + kk) * e.zrs + (int64_t)(c0 + j) * e.zcs] : (TA)0;
        }
        __syncthreads();
        if (tx < qcols) {
          TA sacc[4] = {0, 0, 0, 0};
          for (int kk = 0; kk < pc; ++kk) {
            const TA z = Zs[kk][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (ty + 8 * i < mrows) sacc[i] = fma(Ts[ty + 8 * i][kk], z, sacc[i]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] = fma(f, sacc[i], acc[i]);
        }
        __syncthreads();
      }
    }
  }
  double *D = const_cast<double *>(tptr<double>(db, g.d));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ty + 8 * i;
    if (r < mrows && tx < qcols) D[(int64_t)(r0 + r) * g.drs + (int64_t)(c0 + tx) * g.dcs] += (double)acc[i];
  }
}

// Output blocks of at most 32 x 32: one warp per (output block, entry chunk);
// lanes are assigned to the m*p elements of T = X Y and the m*q elements of
// the output block in flattened order, so a lane is idle only in the last
// partial round (no 32-wide padding of small sector blocks).  Four elements
// per lane are advanced together for instruction-level parallelism.
template <typename TX, typename TY, typename TZ, typename TA, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) chain_flat_kernel(const ChainEntry *__restrict__ E,
                                                               const ChainGroup *__restrict__ G,
                                                               int ngroups, uint64_t xb, uint64_t yb,
                                                               uint64_t zb, uint64_t db) {
  extern __shared__ __align__(16) unsigned char flat_smem[];
  TA *base = reinterpret_cast<TA *>(flat_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = blockIdx.x * WARPS + warp;
  if (gi >= ngroups) return;  // warp-uniform; only warp barriers below
  // three 32 x 33 tiles per warp; the Z tile reuses the X tile once T is formed
  TA(*Xs)[33] = reinterpret_cast<TA(*)[33]>(base + (size_t)warp * 3 * 32 * 33);
  TA(*Ys)[33] = Xs + 32;
  TA(*Ts)[33] = Xs + 64;
  TA(*Zs)[33] = Xs;
  const ChainGroup g = G[gi];
  const int m = g.m, q = g.q, mq = m * q;
  TA acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0;
  for (int ei = g.first; ei < g.first + g.count; ++ei) {
    const ChainEntry e = E[ei];
    const bool xid = e.x == IDN, yid = e.y == IDN, zid = e.z == IDN;
    const TX *X = xid ? nullptr : tptr<TX>(xb, e.x);
    const TY *Y = yid ? nullptr : tptr<TY>(yb, e.y);
    const TZ *Z = zid ? nullptr : tptr<TZ>(zb, e.z);
    const TA f = (TA)e.f;
    const int n = e.n, p = e.p;
    for (int p0 = 0; p0 < p; p0 += 32) {
      const int pc = min(32, p - p0);
      const int mp = m * pc;
      // ---- T (m x pc) into Ts
      if (xid || yid) {
        for (int t = lane; t < mp; t += 32) {
          const int i = t / pc, c = t % pc;
          TA v;
          if (xid && yid) v = (i == p0 + c) ? (TA)1 : (TA)0;
          else if (xid) v = (TA)Y[(int64_t)i * e.yrs + (int64_t)(p0 + c) * e.ycs];
          else v = (TA)X[(int64_t)i * e.xrs + (int64_t)(p0 + c) * e.xcs];
          Ts[i][c] = v;
        }
      } else {
        for (int t = lane; t < mp; t += 32) Ts[t / pc][t % pc] = 0;
        for (int n0 = 0; n0 < n; n0 += 32) {
          const int nc = min(32, n - n0);
          for (int t = lane; t < m * nc; t += 32) {
            const int i = t / nc, kk = t % nc;
            Xs[i][kk] = (TA)X[(int64_t)i * e.xrs + (int64_t)(n0 + kk) * e.xcs];
          }
          for (int t = lane; t < nc * pc; t += 32) {
            const int kk = t / pc, c = t % pc;
            Ys[kk][c] = (TA)Y[(int64_t)(n0 + kk) * e.yrs + (int64_t)(p0 + c) * e.ycs];
          }
          __syncwarp();
          // element t = b0 + 32 u + lane; rounds of four warp-wide element groups
          for (int b0 = 0; b0 < mp; b0 += 128) {
            const int nu = min(4, (mp - b0 + 31) >> 5);  // warp-uniform
            int ii[4], cc[4];
            TA s4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int t = min(b0 + 32 * u + lane, mp - 1);
              ii[u] = t / pc;
              cc[u] = t % pc;
              s4[u] = 0;
            }
            for (int kk = 0; kk < nc; ++kk) {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (u < nu) s4[u] = fma(Xs[ii[u]][kk], Ys[kk][cc[u]], s4[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (b0 + 32 * u + lane < mp) Ts[ii[u]][cc[u]] += s4[u];
          }
          __syncwarp();
        }
      }
      __syncwarp();
      // ---- acc += f T Z (or f T when Z is the identity)
      if (zid) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int t = lane + 32 * j;
          if (t < mq) {
            const int i = t / q, c = t % q;
            if (c >= p0 && c < p0 + pc) acc[j] = fma(f, Ts[i][c - p0], acc[j]);
          }
        }
      } else {
        for (int t = lane; t < pc * q; t += 32) {
          const int kk = t / q, c = t % q;
          Zs[kk][c] = (TA)Z[(int64_t)(p0 + kk) * e.zrs + (int64_t)c * e.zcs];
        }
        __syncwarp();
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 4) {
          const int nu = min(4, (mq - 32 * j0 + 31) >> 5);  // warp-uniform
          if (nu <= 0) break;
          int ii[4], cc[4];
          TA s4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = min(lane + 32 * (j0 + u), mq - 1);
            ii[u] = t / q;
            cc[u] = t % q;
            s4[u] = 0;
          }
          for (int kk = 0; kk < pc; ++kk) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u < nu) s4[u] = fma(Ts[ii[u]][kk], Zs[kk][cc[u]], s4[u]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[j0 + u] = fma(f, s4[u], acc[j0 + u]);
        }
      }
      __syncwarp();
    }
  }
  double *D = const_cast<double *>(tptr<double>(db, g.d));
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int t = lane + 32 * j;
    if (t < mq) D[(int64_t)(t / q) * g.drs + (int64_t)(t % q) * g.dcs] += (double)acc[j];
  }
}

template <typename TX, typename TY, typename TZ, typename TA, int WARPS>
static cudaError_t launch_flat_w(const ChainEntry *e, const ChainGroup *g, int ngroups, uint64_t xb,
                                 uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s) {
  const int smem = WARPS * 3 * 32 * 33 * (int)sizeof(TA);
  auto kern = chain_flat_kernel<TX, TY, TZ, TA, WARPS>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  COUNT(1);
  kern<<<(ngroups + WARPS - 1) / WARPS, 32 * WARPS, smem, s>>>(e, g, ngroups, xb, yb, zb, db);
  return cudaGetLastError();
}

// warps per CTA: FP64 6 (one CTA per SM) or 4 (two CTAs, 8 warps per SM);
// FP32 12 (one CTA) or 8 (two CTAs, 16 warps per SM)
cudaError_t launch_chain_flat_fp64(const ChainEntry *e, const ChainGroup *g, int ngroups, uint64_t xb,
                                   uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s, int warps) {
  if (ngroups <= 0) return cudaSuccess;
  if (warps == 4) return launch_flat_w<double, double, double, double, 4>(e, g, ngroups, xb, yb, zb, db, s);
  return launch_flat_w<double, double, double, double, 6>(e, g, ngroups, xb, yb, zb, db, s);
}

cudaError_t launch_chain_flat_f32ops(const ChainEntry *e, const ChainGroup *g, int ngroups, uint64_t xb,
                                     uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s, int warps) {
  if (ngroups <= 0) return cudaSuccess;
  if (warps == 8) return launch_flat_w<float, double, float, float, 8>(e, g, ngroups, xb, yb, zb, db, s);
  return launch_flat_w<float, double, float, float, 12>(e, g, ngroups, xb, yb, zb, db, s);
}

// out[ red.d + ...] += sum over the task chunks of their partial blocks, in chunk order
__global__ void reduce_partials_kernel(const ReduceGroup *__restrict__ R, int nred, int64_t total,
                                       const double *__restrict__ scratch, double *out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nred - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (R[mid].e0 <= t) lo = mid; else hi = mid - 1;
    }
    const ReduceGroup r = R[lo];
    const int64_t loc = t - r.e0;
    const int i = (int)(loc / r.q), c = (int)(loc % r.q);
    const int64_t mq = (int64_t)r.m * r.q;
    double s = 0.0;
    for (int k = 0; k < r.nsplit; ++k) s += scratch[r.soff + k * mq + loc];
    out[r.d + (int64_t)i * r.drs + (int64_t)c * r.dcs] += s;
  }
}

cudaError_t launch_reduce_partials(const ReduceGroup *r, int nred, int64_t total, const double *scratch,
                                   double *out, cudaStream_t s) {
  if (nred <= 0 || total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  COUNT(1);
  reduce_partials_kernel<<<(int)blocks, 256, 0, s>>>(r, nred, total, scratch, out);
  return cudaGetLastError();
}

cudaError_t launch_chain_fp64(const ChainEntry *e, const ChainGroup *g, int ngroups, int ntiles,
                              uint64_t xb, uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s) {
  if (ngroups <= 0 || ntiles <= 0) return cudaSuccess;
  COUNT(1);
  chain_kernel<double, double, double, double><<<ntiles, 256, 0, s>>>(e, g, ngroups, xb, yb, zb, db);
  return cudaGetLastError();
}

cudaError_t launch_chain_f32ops(const ChainEntry *e, const ChainGroup *g, int ngroups, int ntiles,
                                uint64_t xb, uint64_t yb, uint64_t zb, uint64_t db, cudaStream_t s) {
  if (ngroups <= 0 || ntiles <= 0) return cudaSuccess;
  COUNT(1);
  chain_kernel<float, double, float, float><<<ntiles, 256, 0, s>>>(e, g, ngroups, xb, yb, zb, db);
  return cudaGetLastError();
}

__global__ void to_f32_kernel(float *out, const double *in, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

__global__ void __launch_bounds__(256) lincomb_fp64_kernel(const LincombTask *__restrict__ T,
                                                           int ntasks) {
  __shared__ double Cs[32][33];
  __shared__ double Ss[32][33];
  const int tile = blockIdx.x;
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  const LincombTask t = T[lo];
  const int64_t E = (int64_t)t.rows * t.cols;
  const int ne = (int)((E + 31) / 32);
  const int tl = tile - t.tile0;
  const int t0 = (tl / ne) * 32;
  const int64_t e0 = (int64_t)(tl % ne) * 32;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const double *coef = dptr(0, t.coef);
  const double *src = dptr(0, t.src);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int u0 = 0; u0 < t.ksrc; u0 += 32) {
    for (int idx = tid; idx < 1024; idx += 256) {
      const int i = idx >> 5, j = idx & 31;
      Cs[i][j] = (t0 + i < t.kout && u0 + j < t.ksrc) ? coef[(int64_t)(t0 + i) * t.ksrc + u0 + j] : 0.0;
      const int64_t e = e0 + j;
      double v = 0.0;
      if (u0 + i < t.ksrc && e < E) {
        int64_t se = e;
        if (t.tr) {
          const int64_t r = e / t.cols, c = e % t.cols;
          se = c * t.rows + r;
        }
        v = src[(int64_t)(u0 + i) * E + se];
      }
      Ss[i][j] = v;
    }
    __syncthreads();
    const int uc = min(32, t.ksrc - u0);
    for (int uu = 0; uu < uc; ++uu) {
      const double sv = Ss[uu][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fma(Cs[ty + 8 * i][uu], sv, acc[i]);
    }
    __syncthreads();
  }
  double *out = const_cast<double *>(dptr(0, t.out));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int tt = t0 + ty + 8 * i;
    const int64_t e = e0 + tx;
    if (tt < t.kout && e < E) out[(int64_t)tt * E + e] = acc[i];
  }
}

static int grid_for(int64_t n);

cudaError_t launch_to_f32(float *out, const double *in, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  COUNT(1);
  to_f32_kernel<<<grid_for(n), 256, 0, s>>>(out, in, n);
  return cudaGetLastError();
}

cudaError_t launch_lincomb_fp64(const LincombTask *t, int ntasks, int ntiles, cudaStream_t s) {
  if (ntasks <= 0 || ntiles <= 0) return cudaSuccess;
  COUNT(1);
  lincomb_fp64_kernel<<<ntiles, 256, 0, s>>>(t, ntasks);
  return cudaGetLastError();
}

// diag(H_eff): entries whose input block is their output block contribute f X_ii Z_jj.
__global__ void diag_fp64_kernel(const ChainEntry *__restrict__ E, const ChainGroup *__restrict__ G,
                                 uint64_t xb, uint64_t zb, double *diag) {
  const ChainGroup g = G[blockIdx.x];
  for (int ei = g.first; ei < g.first + g.count; ++ei) {
    const ChainEntry e = E[ei];
    if (e.y != g.d) continue;
    const bool xid = e.x == IDN, zid = e.z == IDN;
    const double *X = xid ? nullptr : dptr(xb, e.x);
    const double *Z = zid ? nullptr : dptr(zb, e.z);
    for (int idx = threadIdx.x; idx < g.m * g.q; idx += blockDim.x) {
      const int i = idx / g.q, j = idx % g.q;
      const double x = xid ? 1.0 : X[(int64_t)i * e.xrs + (int64_t)i * e.xcs];
      const double z = zid ? 1.0 : Z[(int64_t)j * e.zrs + (int64_t)j * e.zcs];
      diag[g.d + (int64_t)i * g.drs + (int64_t)j * g.dcs] += e.f * x * z;
    }
    __syncthreads();
  }
}

cudaError_t launch_diag_fp64(const ChainEntry *e, const ChainGroup *g, int ngroups, uint64_t xb,
                             uint64_t zb, double *diag, cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  COUNT(1);
  diag_fp64_kernel<<<ngroups, 256, 0, s>>>(e, g, xb, zb, diag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Davidson helpers

int dots_partial_blocks(int64_t n) {
  int64_t b = (n + 2047) / 2048;
  if (b < 1) b = 1;
  if (b > 608) b = 608;  // 4 per SM on 152 SMs
  return (int)b;
}

__global__ void dots_stage1(const double *__restrict__ V, int k, int64_t n,
                            const double *__restrict__ w, double *partial) {
  __shared__ double red[32][33];
  const int nb = gridDim.x;
  double s[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) s[j] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)nb * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < k) s[j] = fma(V[(int64_t)j * n + e], we, s[j]);
  }
  // warp reduce
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    double x = s[j];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double x = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) x += red[w2][threadIdx.x];
    partial[(int64_t)blockIdx.x * k + threadIdx.x] = x;
  }
}

__global__ void dots_stage2(const double *partial, int nb, int k, double *out) {
  const int j = blockIdx.x;
  __shared__ double red[256];
  double x = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) x += partial[(int64_t)b * k + j];
  red[threadIdx.x] = x;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

cudaError_t launch_dots(const double *V, int k, int64_t n, const double *w, double *partial,
                        double *out, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const int nb = dots_partial_blocks(n);
  COUNT(1);
  dots_stage1<<<nb, 256, 0, s>>>(V, k, n, w, partial);
  COUNT(1);
  dots_stage2<<<k, 256, 0, s>>>(partial, nb, k, out);
  return cudaGetLastError();
}

__global__ void combine_kernel(double *out, const double *__restrict__ V, const double *__restrict__ y,
                               int k, int64_t n, double beta) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = beta == 0.0 ? 0.0 : beta * out[e];
    for (int j = 0; j < k; ++j) s = fma(y[j], V[(int64_t)j * n + e], s);
    out[e] = s;
  }
}

static int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_combine(double *out, const double *V, const double *y, int k, int64_t n,
                           double beta, cudaStream_t s) {
  COUNT(1);
  combine_kernel<<<grid_for(n), 256, 0, s>>>(out, V, y, k, n, beta);
  return cudaGetLastError();
}

__global__ void sub_proj_kernel(double *w, const double *__restrict__ V, const double *__restrict__ c,
                                int k, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = w[e];
    for (int j = 0; j < k; ++j) s = fma(-c[j], V[(int64_t)j * n + e], s);
    w[e] = s;
  }
}

cudaError_t launch_sub_proj(double *w, const double *V, const double *c, int k, int64_t n,
                            cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  COUNT(1);
  sub_proj_kernel<<<grid_for(n), 256, 0, s>>>(w, V, c, k, n);
  return cudaGetLastError();
}

__global__ void axpy_kernel(double *y, const double *x, double a, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

cudaError_t launch_axpy(double *y, const double *x, double a, int64_t n, cudaStream_t s) {
  COUNT(1);
  axpy_kernel<<<grid_for(n), 256, 0, s>>>(y, x, a, n);
  return cudaGetLastError();
}

__global__ void scale_kernel(double *x, const double *a_dev, int invert_sqrt, int64_t n) {
  const double a = invert_sqrt ? 1.0 / sqrt(*a_dev) : *a_dev;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] *= a;
}

cudaError_t launch_scale(double *x, const double *a_dev, int invert_sqrt, int64_t n, cudaStream_t s) {
  COUNT(1);
  scale_kernel<<<grid_for(n), 256, 0, s>>>(x, a_dev, invert_sqrt, n);
  return cudaGetLastError();
}

__global__ void precond_kernel(double *t, const double *r, const double *diag, const double *theta,
                               int64_t n) {
  const double th = *theta;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double d = th - diag[e];
    if (fabs(d) < 1e-8) d = d < 0.0 ? -1e-8 : 1e-8;
    t[e] = r[e] / d;
  }
}

cudaError_t launch_precond(double *t, const double *r, const double *diag, const double *theta,
                           int64_t n, cudaStream_t s) {
  COUNT(1);
  precond_kernel<<<grid_for(n), 256, 0, s>>>(t, r, diag, theta, n);
  return cudaGetLastError();
}

__global__ void residual_kernel(double *r, const double *hx, const double *x, const double *theta,
                                int64_t n) {
  const double th = *theta;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    r[e] = fma(-th, x[e], hx[e]);
}

cudaError_t launch_residual(double *r, const double *hx, const double *x, const double *theta,
                            int64_t n, cudaStream_t s) {
  COUNT(1);
  residual_kernel<<<grid_for(n), 256, 0, s>>>(r, hx, x, theta, n);
  return cudaGetLastError();
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_guess_kernel(double *x, int64_t n, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed * 0x100000001B3ull + (uint64_t)e);
    x[e] = 2.0 * ((double)(r >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  }
}

cudaError_t launch_fill_guess(double *x, int64_t n, uint64_t seed, cudaStream_t s) {
  COUNT(1);
  fill_guess_kernel<<<grid_for(n), 256, 0, s>>>(x, n, seed);
  return cudaGetLastError();
}

// Symmetric eigensolver for the small Davidson subspace matrix (n <= 32):
// two-sided Jacobi with the round-robin (circle) ordering, so each round
// applies n/2 disjoint rotations at once (they commute), one thread per pair
// for the angles and one thread per (row, pair) for the updates.  Rotation
// angles as in the classical cyclic method (t = sgn(th)/(|th|+sqrt(th^2+1)),
// th = (a_qq - a_pp)/(2 a_pq)); sweeps until the off-diagonal norm is below
// 1e-16 of the diagonal norm.  Eigenvalues ascending; evecs row-major with
// eigenvector j in column j.
__global__ void __launch_bounds__(128) jacobi_eigh_kernel(const double *A, int n, int lda, double *evals,
                                                          double *evecs) {
  __shared__ double a[32][33];
  __shared__ double v[32][33];
  __shared__ double rc[16], rs[16];
  __shared__ int rp[16], rq[16];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    a[i][j] = A[(int64_t)i * lda + j];
    v[i][j] = (i == j) ? 1.0 : 0.0;
  }
  const int N = (n + 1) & ~1;  // an odd n gets a dummy index n (its pairs are skipped)
  const int npair = N / 2;
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid < 32) {
      double off = 0.0, dg = 0.0;
      if (tid < n) {
        dg = a[tid][tid] * a[tid][tid];
        for (int j = tid + 1; j < n; ++j) off += a[tid][j] * a[tid][j];
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dg += __shfl_xor_sync(0xffffffffu, dg, o);
      }
      if (tid == 0) done = off <= 1e-32 * (dg + 1e-300);
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < N - 1; ++r) {
      if (tid < npair) {
        const int i0 = tid, i1 = N - 1 - tid;
        int p = i0 == 0 ? 0 : ((i0 - 1 + r) % (N - 1)) + 1;
        int q = ((i1 - 1 + r) % (N - 1)) + 1;
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        double c = 1.0, sn = 0.0;
        if (q < n) {
          const double apq = a[p][q];
          if (fabs(apq) >= 1e-300) {
            const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sn = t * c;
          }
        } else {
          p = -1;
        }
        rp[tid] = p;
        rq[tid] = q;
        rc[tid] = c;
        rs[tid] = sn;
      }
      __syncthreads();
      for (int it = tid; it < n * npair; it += nt) {  // A <- A J, V <- V J
        const int k = it % n, m = it / n, p = rp[m], q = rq[m];
        if (p < 0) continue;
        const double c = rc[m], sn = rs[m];
        const double akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - sn * akq;
        a[k][q] = sn * akp + c * akq;
        const double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - sn * vkq;
        v[k][q] = sn * vkp + c * vkq;
      }
      __syncthreads();
      for (int it = tid; it < n * npair; it += nt) {  // A <- J^T A
        const int k = it % n, m = it / n, p = rp[m], q = rq[m];
        if (p < 0) continue;
        const double c = rc[m], sn = rs[m];
        const double apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - sn * aqk;
        a[q][k] = sn * apk + c * aqk;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int i = 0; i < n; ++i) {
      int m = i;
      for (int j = i + 1; j < n; ++j)
        if (a[j][j] < a[m][m]) m = j;
      if (m != i) {
        const double t = a[i][i];
        a[i][i] = a[m][m];
        a[m][m] = t;
        for (int r = 0; r < n; ++r) {
          const double x = v[r][i];
          v[r][i] = v[r][m];
          v[r][m] = x;
        }
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) evecs[idx] = v[idx / n][idx % n];
  if (tid < n) evals[tid] = a[tid][tid];
}

cudaError_t launch_jacobi_eigh(const double *A, int n, int lda, double *evals, double *evecs,
                               cudaStream_t s) {
  if (n > 32 || n < 1) return cudaErrorInvalidValue;
  COUNT(1);
  jacobi_eigh_kernel<<<1, 128, 0, s>>>(A, n, lda, evals, evecs);
  return cudaGetLastError();
}

// O[i][c] = evecs[:, cols[c]][i] for column-major evecs (n x n)
__global__ void gather_columns_kernel(double *O, const double *evecs, int n, const int *cols, int kept) {
  const int64_t tot = (int64_t)n * kept;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / kept, c = idx % kept;
    O[idx] = evecs[(int64_t)cols[c] * n + i];
  }
}

cudaError_t launch_gather_columns(double *O, const double *evecs, int n, const int *cols, int kept,
                                  cudaStream_t s) {
  if (kept <= 0 || n <= 0) return cudaSuccess;
  COUNT(1);
  gather_columns_kernel<<<grid_for((int64_t)n * kept), 256, 0, s>>>(O, evecs, n, cols, kept);
  return cudaGetLastError();
}

}  // namespace dmrg
