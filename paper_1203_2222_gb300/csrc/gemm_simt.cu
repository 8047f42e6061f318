// Grouped per-sector GEMM on the CUDA cores, FP64 or exact FP32.
//
// Blockwise matrix multiply of Ch. 5, Eq. blockmult, T_j = M_j N_j, for
// every sector j of a contraction in one launch.  It is the whole GEMM of the
// plain FP64 path and, in the split-BF16 path, the kernel for sectors whose
// matrices are too thin to fill a 128 x 128 tensor-core tile (tiny k, or
// n <= 16) -- those are bandwidth-bound and are computed here in FP32.
//
// One CTA of 256 threads per output tile (TM x TN, each thread a
// (TM/16) x (TN/16) register tile), 16-deep k slices staged in shared
// memory.  A tile may cover only a slice [k0, k1) of the reduction: the
// planner splits long reductions with few output tiles across CTAs, which
// then add into a zero-filled C with atomics.
#include <cuda_runtime.h>

#include "kernels.h"

namespace sym {
namespace {

constexpr int KS = 16;

template <typename T, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const GemmSectorSimt* __restrict__ secs,
                                                        const GemmTile* __restrict__ tiles,
                                                        const T* __restrict__ ops, T* __restrict__ outm) {
  constexpr int RM = TM / 16, RN = TN / 16;
  __shared__ T As[KS][TM + 1];
  __shared__ T Bs[KS][TN];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmSectorSimt s = secs[tl.sector];
  const int m0 = tl.mt * TM, n0 = tl.nt * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = T(0);
  const T* a = ops + s.a_off;
  const T* b = ops + s.b_off;
  for (int kb = tl.k0; kb < tl.k1; kb += KS) {
    for (int i = threadIdx.x; i < TM * KS; i += 256) {
      const int r = i / KS, c = i % KS;
      const int gr = m0 + r, gc = kb + c;
      As[c][r] = (gr < s.m && gc < tl.k1) ? a[(int64_t)gr * s.lda + gc] : T(0);
    }
    for (int i = threadIdx.x; i < TN * KS; i += 256) {
      const int r = i / TN, c = i % TN;
      const int gr = kb + r, gc = n0 + c;
      Bs[r][c] = (gr < tl.k1 && gc < s.n) ? b[(int64_t)gr * s.ldb + gc] : T(0);
    }
    __syncthreads();
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

template <typename T>
int launch_t(int shape, const GemmSectorSimt* secs, const GemmTile* tiles, int ntiles, const void* ops, void* outm,
             cudaStream_t s) {
  const T* o = static_cast<const T*>(ops);
  T* c = static_cast<T*>(outm);
  if (shape == SIMT_64x64)
    gemm_simt_kernel<T, 64, 64><<<ntiles, 256, 0, s>>>(secs, tiles, o, c);
  else
    gemm_simt_kernel<T, 256, 16><<<ntiles, 256, 0, s>>>(secs, tiles, o, c);
  return (int)cudaGetLastError();
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
