// Plain FP64 grouped GEMM on the CUDA cores: the FP64 comparator path.
//
// Blockwise matrix multiply of Ch. 5, Eq. blockmult, T_j = M_j N_j, for every
// sector j of a contraction in one launch.  One CTA per 64 x 64 output tile
// (tile list precomputed on the host, largest k first); 256 threads, each a
// 4 x 4 register tile; 16-deep k slices staged in shared memory.
#include <cuda_runtime.h>

#include "kernels.h"

namespace sym {
namespace {

constexpr int T = 64, KS = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmSector64* __restrict__ secs,
                                                       const GemmTile* __restrict__ tiles,
                                                       const double* __restrict__ A,
                                                       const double* __restrict__ B, double* __restrict__ C) {
  __shared__ double As[KS][T + 1];
  __shared__ double Bs[KS][T];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmSector64 s = secs[tl.sector];
  const int m0 = tl.mt * T, n0 = tl.nt * T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const double* a = A + s.a_off;
  const double* b = B + s.b_off;
  for (int k0 = 0; k0 < s.k; k0 += KS) {
    for (int i = threadIdx.x; i < T * KS; i += 256) {
      int r = i / KS, c = i % KS;
      int gr = m0 + r, gc = k0 + c;
      As[c][r] = (gr < s.m && gc < s.k) ? a[(int64_t)gr * s.lda + gc] : 0.0;
    }
    for (int i = threadIdx.x; i < T * KS; i += 256) {
      int r = i / T, c = i % T;
      int gr = k0 + r, gc = n0 + c;
      Bs[r][c] = (gr < s.k && gc < s.n) ? b[(int64_t)gr * s.ldb + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* c = C + s.c_off;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + ty + 16 * i;
    if (r >= s.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int cc = n0 + tx + 16 * j;
      if (cc < s.n) c[(int64_t)r * s.ldc + cc] = s.alpha * acc[i][j];
    }
  }
}

}  // namespace

int launch_gemm_f64(const GemmSector64* secs, const GemmTile* tiles, int ntiles, const double* A, const double* B,
                    double* C, void* stream) {
  if (ntiles <= 0) return 0;
  gemm_f64_kernel<<<ntiles, 256, 0, static_cast<cudaStream_t>(stream)>>>(secs, tiles, A, B, C);
  return (int)cudaGetLastError();
}

}  // namespace sym
