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
//   rows  k, n <= 16: a persistent streaming kernel -- each warp stages runs
//         of whole rows of A in shared memory and writes whole rows of C.
//   thin  m, n <= 8 and a long reduction: each thread streams k and keeps
//         the whole m x n outer-product sum in registers, then the CTA
//         reduces and adds its slice into C.
#include <cuda_runtime.h>

#include <algorithm>

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

// k, n <= 16: C = A B streamed.  Persistent: each warp walks its own tiles
// (row ranges of one sector).  Per step it reads rows_span(k) whole rows of
// A -- one contiguous run of <= 512 elements -- with coalesced loads into its
// shared-memory span (the next run is in flight in registers meanwhile);
// then lane (rl, j) = (lane >> lg, lane & (2^lg - 1)), 2^lg >= n, computes
// C[r, j] for rows r = rl, rl + 32 >> lg, ... of the run, with its column of
// B in registers, so each store instruction writes whole consecutive rows of
// C.  A and C are dense (lda == k, ldc == n); B may be stored transposed.
template <typename T>
__global__ void __launch_bounds__(256) gemm_rows_kernel(const GemmSectorSimt* __restrict__ secs,
                                                        const GemmTile* __restrict__ tiles, int ntiles,
                                                        const T* __restrict__ ops, T* __restrict__ outm) {
  constexpr int V = kRowsSpan / 32;  // elements of a run per lane
  __shared__ T span[8][kRowsSpan];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* __restrict__ sp = span[warp];
  pdl_wait();
  pdl_launch_dependents();
  for (int t = blockIdx.x * 8 + warp; t < ntiles; t += gridDim.x * 8) {
    const GemmTile tl = tiles[t];
    const GemmSectorSimt s = secs[tl.sector];
    const int k = s.k, n = s.n;
    const int lg = n <= 1 ? 0 : n <= 2 ? 1 : n <= 4 ? 2 : n <= 8 ? 3 : 4;
    const int j = lane & ((1 << lg) - 1), rl = lane >> lg, rstep = 32 >> lg;
    const int rw = rows_span(k);
    const T* __restrict__ a = ops + s.a_off;
    const T* __restrict__ b = ops + s.b_off;
    T* __restrict__ c = outm + s.c_off;
    const int64_t bj = (s.trans & kTransB) ? (int64_t)j * s.ldb : j, bk = (s.trans & kTransB) ? 1 : s.ldb;
    T bv[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) bv[kk] = (kk < k && j < n) ? __ldg(b + bj + kk * bk) : T(0);
    const T alpha = T(s.alpha);
    T v[V];
    auto load = [&](int r0) {
      const int lim = min(rw, tl.k1 - r0) * k;  // elements of this run
      const T* __restrict__ src = a + (int64_t)r0 * k;
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int e = lane + 32 * u;
        v[u] = e < lim ? __ldg(src + e) : T(0);
      }
    };
    load(tl.k0);
    for (int r0 = tl.k0; r0 < tl.k1; r0 += rw) {
      __syncwarp();  // the previous run's readers are done with the span
#pragma unroll
      for (int u = 0; u < V; ++u) sp[lane + 32 * u] = v[u];
      __syncwarp();
      if (r0 + rw < tl.k1) load(r0 + rw);
      const int nr = min(rw, tl.k1 - r0);
      T* __restrict__ cr = c + (int64_t)r0 * n + j;
      for (int rr = rl; rr < nr; rr += rstep) {
        const T* __restrict__ row = sp + rr * k;
        T acc = T(0);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
          if (kk < k) acc = fma(row[kk], bv[kk], acc);
        if (j < n) cr[(int64_t)rr * n] = alpha * acc;
      }
    }
  }
}

// Thin GEMM: m, n <= 8 and a long reduction (e.g. the gradient of a small
// operator).  Each thread streams k values (coalesced along A's rows and
// B's short rows, or through L1 along the short rows of a transposed A) and
// keeps the whole m x n outer-product sum in registers; the CTA then reduces
// across its threads and adds its slice into C.
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
  // element strides of A (i, kk) and B (kk, j), plain or transposed storage
  const int64_t ai = (s.trans & kTransA) ? 1 : s.lda, ak = (s.trans & kTransA) ? s.lda : 1;
  const int64_t bk = (s.trans & kTransB) ? 1 : s.ldb, bj = (s.trans & kTransB) ? s.ldb : 1;
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
      for (int i = 0; i < MX; ++i) av[u][i] = (ok && i < s.m) ? __ldg(a + i * ai + kk * ak) : T(0);
#pragma unroll
      for (int j = 0; j < MX; ++j) bv[u][j] = (ok && j < s.n) ? __ldg(b + kk * bk + j * bj) : T(0);
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

// resident CTAs of the rows kernel per SM (queried once per type)
template <typename T>
int rows_ctas_per_sm() {
  static const int n = [] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_rows_kernel<T>, 256, 0) != cudaSuccess || v < 1) v = 1;
    return v;
  }();
  return n;
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
    default: {
      const int ctas = std::min((ntiles + 7) / 8, tc_num_sms() * rows_ctas_per_sm<T>());
      return (int)launch_pdl(gemm_rows_kernel<T>, dim3(ctas), b, 0, s, secs, tiles, ntiles, o, c);
    }
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
