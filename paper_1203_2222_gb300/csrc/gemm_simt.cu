// Grouped per-sector GEMM on the CUDA cores, FP64 or exact FP32.
//
// Blockwise matrix multiply of Ch. 5, Eq. blockmult, T_j = M_j N_j, for
// every sector j of a contraction in one launch.  It is the whole GEMM of the
// plain FP64 path and, in the split-BF16 path, the kernel for sectors whose
// matrices are too thin to fill a 128 x 128 tensor-core tile -- those are
// bandwidth- or latency-bound and are computed here in FP32.
//
// Three kernels, chosen per sector by the planner:
//   tile  TM x TN output tile per 256-thread CTA, 32-deep k slices staged in
//         shared memory, the next slice prefetched into registers while the
//         current one is multiplied; a tile may cover a slice [k0, k1) of the
//         reduction (split-K: slices add into a zero-filled C with atomics).
//   rows  k, n <= 16: one output row per thread, B held in shared memory --
//         a streaming kernel (read a row of A, write a row of C).
//   thin  m, n <= 8 and a long reduction: each thread streams k and keeps
//         the whole m x n outer-product sum in registers, then the CTA
//         reduces and adds its slice into C.
#include <cuda_runtime.h>

#include "kernels.h"
#include "pdl.h"

namespace sym {
namespace {

template <typename T, int TM, int TN, int KS = (TM == 256 && sizeof(T) == 8) ? 16 : 32>
__global__ void __launch_bounds__(256) gemm_tile_kernel(const GemmSectorSimt* __restrict__ secs,
                                                        const GemmTile* __restrict__ tiles,
                                                        const T* __restrict__ ops, T* __restrict__ outm) {
  constexpr int RM = TM / 16, RN = TN / 16;
  constexpr int LA = TM * KS / 256, LB = TN * KS / 256;  // slice elements per thread
  __shared__ T As[KS][TM + 1];
  __shared__ T Bs[KS][TN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmSectorSimt s = secs[tl.sector];
  pdl_wait();
  pdl_launch_dependents();
  const int m0 = tl.mt * TM, n0 = tl.nt * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = T(0);
  const T* __restrict__ a = ops + s.a_off;
  const T* __restrict__ b = ops + s.b_off;
  T ra[LA], rb[LB];
  auto load = [&](int kb) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int i = threadIdx.x + 256 * u;
      const int r = i / KS, c = i % KS;
      const int gr = m0 + r, gc = kb + c;
      ra[u] = (gr < s.m && gc < tl.k1) ? __ldg(a + (int64_t)gr * s.lda + gc) : T(0);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int i = threadIdx.x + 256 * u;
      const int r = i / TN, c = i % TN;
      const int gr = kb + r, gc = n0 + c;
      rb[u] = (gr < tl.k1 && gc < s.n) ? __ldg(b + (int64_t)gr * s.ldb + gc) : T(0);
    }
  };
  load(tl.k0);
  for (int kb = tl.k0; kb < tl.k1; kb += KS) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int i = threadIdx.x + 256 * u;
      As[i % KS][i / KS] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int i = threadIdx.x + 256 * u;
      Bs[i / TN][i % TN] = rb[u];
    }
    __syncthreads();
    if (kb + KS < tl.k1) load(kb + KS);  // next slice in flight during the multiply
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      T av[RM], bv[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* c = outm + s.c_off;
  const T alpha = T(s.alpha);
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= s.m) continue;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int cc = n0 + tx + 16 * j;
      if (cc >= s.n) continue;
      if (tl.atomic)
        atomicAdd(&c[(int64_t)r * s.ldc + cc], alpha * acc[i][j]);
      else
        c[(int64_t)r * s.ldc + cc] = alpha * acc[i][j];
    }
  }
}

// k, n <= 16: C[r, :] = A[r, :] B, one row per thread, 256 rows per CTA.
template <typename T>
__global__ void __launch_bounds__(256) gemm_rows_kernel(const GemmSectorSimt* __restrict__ secs,
                                                        const GemmTile* __restrict__ tiles,
                                                        const T* __restrict__ ops, T* __restrict__ outm) {
  __shared__ T Bs[16][17];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmSectorSimt s = secs[tl.sector];
  pdl_wait();
  pdl_launch_dependents();
  const T* __restrict__ a = ops + s.a_off;
  const T* __restrict__ b = ops + s.b_off;
  for (int i = threadIdx.x; i < s.k * s.n; i += 256) Bs[i / s.n][i % s.n] = __ldg(b + (int64_t)(i / s.n) * s.ldb + i % s.n);
  __syncthreads();
  const int r = tl.mt * 256 + threadIdx.x;
  if (r >= s.m) return;
  T av[16];
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) av[kk] = kk < s.k ? __ldg(a + (int64_t)r * s.lda + kk) : T(0);
  T* c = outm + s.c_off + (int64_t)r * s.ldc;
  const T alpha = T(s.alpha);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j >= s.n) break;
    T acc = T(0);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
      if (kk < s.k) acc = fma(av[kk], Bs[kk][j], acc);
    c[j] = alpha * acc;
  }
}

// Thin GEMM: m, n <= 8 and a long reduction (e.g. the gradient of a small
// operator).  Each thread streams k values (coalesced along A's rows and
// B's short rows) and keeps the whole m x n outer-product sum in registers;
// the CTA then reduces across its threads and adds its slice into C.
template <typename T>
__global__ void __launch_bounds__(256) gemm_thin_kernel(const GemmSectorSimt* __restrict__ secs,
                                                        const GemmTile* __restrict__ tiles,
                                                        const T* __restrict__ ops, T* __restrict__ outm) {
  constexpr int MX = 8, U = 4;
  __shared__ T red[8][MX * MX];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmSectorSimt s = secs[tl.sector];
  pdl_wait();
  pdl_launch_dependents();
  const T* __restrict__ a = ops + s.a_off;
  const T* __restrict__ b = ops + s.b_off;
  T acc[MX][MX];
#pragma unroll
  for (int i = 0; i < MX; ++i)
#pragma unroll
    for (int j = 0; j < MX; ++j) acc[i][j] = T(0);
  for (int k = tl.k0 + threadIdx.x; k < tl.k1; k += 256 * U) {
    T av[U][MX], bv[U][MX];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int kk = k + 256 * u;
      const bool ok = kk < tl.k1;
#pragma unroll
      for (int i = 0; i < MX; ++i) av[u][i] = (ok && i < s.m) ? __ldg(a + (int64_t)i * s.lda + kk) : T(0);
#pragma unroll
      for (int j = 0; j < MX; ++j) bv[u][j] = (ok && j < s.n) ? __ldg(b + (int64_t)kk * s.ldb + j) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int i = 0; i < MX; ++i)
#pragma unroll
        for (int j = 0; j < MX; ++j) acc[i][j] = fma(av[u][i], bv[u][j], acc[i][j]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MX; ++i)
#pragma unroll
    for (int j = 0; j < MX; ++j) {
      T v = acc[i][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i * MX + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < MX * MX) {
    const int i = threadIdx.x / MX, j = threadIdx.x % MX;
    if (i < s.m && j < s.n) {
      T v = T(0);
#pragma unroll
      for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
      v *= T(s.alpha);
      T* c = outm + s.c_off + (int64_t)i * s.ldc + j;
      if (tl.atomic)
        atomicAdd(c, v);
      else
        *c = v;
    }
  }
}

template <typename T>
int launch_t(int shape, const GemmSectorSimt* secs, const GemmTile* tiles, int ntiles, const void* ops, void* outm,
             cudaStream_t s) {
  const T* o = static_cast<const T*>(ops);
  T* c = static_cast<T*>(outm);
  const dim3 g(ntiles), b(256);
  switch (shape) {
    case SIMT_64x64: return (int)launch_pdl(gemm_tile_kernel<T, 64, 64>, g, b, 0, s, secs, tiles, o, c);
    case SIMT_256x16: return (int)launch_pdl(gemm_tile_kernel<T, 256, 16>, g, b, 0, s, secs, tiles, o, c);
    case SIMT_THIN: return (int)launch_pdl(gemm_thin_kernel<T>, g, b, 0, s, secs, tiles, o, c);
    default: return (int)launch_pdl(gemm_rows_kernel<T>, g, b, 0, s, secs, tiles, o, c);
  }
}

}  // namespace

int launch_gemm_simt(bool f64, int shape, const GemmSectorSimt* secs, const GemmTile* tiles, int ntiles,
                     const void* ops, void* outm, void* stream) {
  if (ntiles <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return f64 ? launch_t<double>(shape, secs, tiles, ntiles, ops, outm, s)
             : launch_t<float>(shape, secs, tiles, ntiles, ops, outm, s);
}

}  // namespace sym
