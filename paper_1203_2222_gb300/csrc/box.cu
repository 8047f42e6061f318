// Block movement kernel: every permute / fuse / split / matrix-form gather /
// scatter of the library is a set of strided boxes, each destination element
// being a short sum of coefficient x source element (one term for U(1) and
// for pure re-indexing; the recoupling sum of Ch. 6, Eq. permsu2, for SU(2)).
//
// One CTA of 256 threads handles one BoxItem: a chunk of at most 2048
// elements of one box, 8 per thread.  Every thread first computes the offsets
// of its 8 elements (index decomposition by reciprocal multiplication) and
// issues all their loads, then stores them, so a CTA needs a single memory
// round trip after reading its descriptor; the first term of the sum is
// carried in the descriptor itself.  Consecutive threads take consecutive
// elements of the box, whose last dimension the planner makes the source's
// fastest one (coalesced reads).  Memory-bound: bytes = source read +
// destination written.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace sym {
namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 8;
constexpr int kMaxSmemTerms = 64;
constexpr int kItemWords = (int)(sizeof(BoxItem) / 4);
static_assert(sizeof(BoxItem) % 8 == 0, "BoxItem must be a whole number of 8-byte words");

// floor(a / n) for a >= 0: float reciprocal (off by at most one for
// a < 2^22, then corrected), exact integer division beyond
__device__ __forceinline__ int fdiv(int a, int n, float rn) {
  if (a >= (1 << 22)) return a / n;
  int q = __float2int_rz(__int2float_rz(a) * rn);
  const int r = a - q * n;
  q += (r >= n) - (r < 0);
  return q;
}

template <typename TD>
__device__ __forceinline__ void store_elem(const BoxItem& it, void* dst0, void* dst1, bool image, TD v, int da,
                                           int db) {
  if (!image) {
    static_cast<TD*>(dst0)[it.dst_off + (int64_t)it.dst_ld * da + db] = v;
  } else {
    // split-BF16: hi = bf16(v), lo = bf16(v - hi); tiled, 128B-swizzled image
    const float x = (float)v;
    const int row = it.row0 + da;
    const int col = it.col0 + db;
    const int64_t off = it.dst_off + ((int64_t)(row >> 7) * it.dst_ld + (col >> 6)) * 8192 + (row & 127) * 64 +
                        ((((col >> 3) & 7) ^ (row & 7)) << 3) + (col & 7);
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    static_cast<__nv_bfloat16*>(dst0)[off] = hi;
    static_cast<__nv_bfloat16*>(dst1)[off] = lo;
  }
}

template <typename TS, typename TD>
__device__ __forceinline__ TD load_elem(const BoxItem& it, const Term* __restrict__ terms, const int64_t* toff,
                                        const int64_t* tld, const double* tcoef, const TS* __restrict__ src, int sa,
                                        int sb) {
  const int nterm = it.nterm;
  if (nterm == 1) return TD(it.t0_coef) * TD(__ldg(src + it.t0_off + it.t0_ld * sa + sb));
  TD acc = TD(0);
  for (int i = 0; i < nterm; ++i) {
    int64_t off;
    double c;
    if (i < kMaxSmemTerms) {
      off = toff[i] + tld[i] * sa;
      c = tcoef[i];
    } else {
      const Term t = terms[it.term0 + i];
      off = t.off + t.ld * sa;
      c = t.coef;
    }
    acc += TD(c) * TD(__ldg(src + off + sb));
  }
  return acc;
}

// Transposing tile: read 32 x 32 elements along the source-contiguous last
// dim (q), stage them in shared memory, write them along the destination-
// contiguous dim (p) -- both sides coalesced.
template <typename TS, typename TD>
__device__ __noinline__ void tile_path(const BoxItem& it, const float* rcp, const Term* __restrict__ terms,
                                       const int64_t* toff, const int64_t* tld, const double* tcoef,
                                       const TS* __restrict__ src, void* dst0, void* dst1, bool image) {
  __shared__ TD tile[32][33];
  const int nd = it.ndim;
  const int P = it.dims[nd - 2], Q = it.dims[nd - 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps
  for (int o = it.start; o < it.start + it.count; ++o) {
    int rem = o, sa = 0, sb = 0, da = 0, db = 0;
#pragma unroll
    for (int d = kMaxDim - 3; d >= 0; --d) {
      if (d < nd - 2) {
        const int n = it.dims[d];
        const int q = fdiv(rem, n, rcp[d]);
        const int t = rem - q * n;
        rem = q;
        sa += t * it.sa[d];
        sb += t * it.sb[d];
        da += t * it.da[d];
        db += t * it.db[d];
      }
    }
    TD v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = it.p0 + w + 8 * u, q = it.q0 + lane;
      v[u] = (p < P && q < Q) ? load_elem<TS, TD>(it, terms, toff, tld, tcoef, src,
                                                  sa + p * it.sa[nd - 2] + q * it.sa[nd - 1],
                                                  sb + p * it.sb[nd - 2] + q * it.sb[nd - 1])
                              : TD(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) tile[w + 8 * u][lane] = v[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = it.q0 + w + 8 * u, p = it.p0 + lane;
      if (p < P && q < Q)
        store_elem<TD>(it, dst0, dst1, image, tile[lane][w + 8 * u], da + p * it.da[nd - 2] + q * it.da[nd - 1],
                       db + p * it.db[nd - 2] + q * it.db[nd - 1]);
    }
    __syncthreads();
  }
}

// offsets of element e: rolled loop over the dims (descriptor in shared memory)
__device__ __forceinline__ void offsets(const BoxItem& it, const float* rcp, int nd, int e, int& sa, int& sb,
                                        int& da, int& db) {
  int rem = e;
  sa = sb = da = db = 0;
#pragma unroll 1
  for (int d = nd - 1; d >= 0; --d) {
    const int n = it.dims[d];
    const int q = fdiv(rem, n, rcp[d]);
    const int t = rem - q * n;
    rem = q;
    sa += t * it.sa[d];
    sb += t * it.sb[d];
    da += t * it.da[d];
    db += t * it.db[d];
  }
}

template <typename TS, typename TD>
__global__ void __launch_bounds__(kThreads) box_kernel(const BoxItem* __restrict__ items,
                                                          const Term* __restrict__ terms, const BoxPtrs ptrs) {
  __shared__ int64_t raw[kItemWords / 2];
  __shared__ float rcp[kMaxDim];
  __shared__ int64_t toff[kMaxSmemTerms], tld[kMaxSmemTerms];
  __shared__ double tcoef[kMaxSmemTerms];
  const int64_t* g = reinterpret_cast<const int64_t*>(items + blockIdx.x);
  if (threadIdx.x < kItemWords / 2) raw[threadIdx.x] = g[threadIdx.x];
  __syncthreads();
  const BoxItem& it = *reinterpret_cast<const BoxItem*>(raw);
  const int nterm = it.nterm;
  if (threadIdx.x < it.ndim) rcp[threadIdx.x] = 1.0f / (float)it.dims[threadIdx.x];
  if (nterm > 1) {
    for (int i = threadIdx.x; i < nterm && i < kMaxSmemTerms; i += blockDim.x) {
      const Term t = terms[it.term0 + i];
      toff[i] = t.off;
      tld[i] = t.ld;
      tcoef[i] = t.coef;
    }
  }
  __syncthreads();
  const int sslot = it.sel & 3, dslot = (it.sel >> 4) & 7;
  const TS* __restrict__ src = static_cast<const TS*>(sslot == 0   ? ptrs.src[0]
                                                      : sslot == 1 ? ptrs.src[1]
                                                      : sslot == 2 ? ptrs.src[2]
                                                                   : ptrs.src[3]);
  void* dst0;
  void* dst1 = ptrs.dst[0][1];
  switch (dslot) {
    case 0: dst0 = ptrs.dst[0][0]; break;
    case 1: dst0 = ptrs.dst[1][0]; break;
    case 2: dst0 = ptrs.dst[2][0]; break;
    case 3: dst0 = ptrs.dst[3][0]; break;
    case 4: dst0 = ptrs.dst[4][0]; break;
    default: dst0 = ptrs.dst[5][0]; break;
  }
  const bool image = (it.sel & kSelImage) != 0;
  const int nd = it.ndim;
  if (it.sel & kSelTile) {
    tile_path<TS, TD>(it, rcp, terms, toff, tld, tcoef, src, dst0, dst1, image);
    return;
  }
  const int e_end = it.start + it.count;
  TD v[kBatch];
  int dda[kBatch], ddb[kBatch];
#pragma unroll
  for (int u = 0; u < kBatch; ++u) {
    const int e = it.start + threadIdx.x + kThreads * u;
    v[u] = TD(0);
    dda[u] = ddb[u] = 0;
    if (e < e_end) {
      int sa, sb;
      offsets(it, rcp, nd, e, sa, sb, dda[u], ddb[u]);
      v[u] = load_elem<TS, TD>(it, terms, toff, tld, tcoef, src, sa, sb);
    }
  }
#pragma unroll
  for (int u = 0; u < kBatch; ++u) {
    const int e = it.start + threadIdx.x + kThreads * u;
    if (e < e_end) store_elem<TD>(it, dst0, dst1, image, v[u], dda[u], ddb[u]);
  }
}

}  // namespace

int launch_box(bool src_f64, bool dst_f64, const BoxItem* items, int nitems, const Term* terms, const BoxPtrs& ptrs,
               void* stream) {
  if (nitems <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid(nitems), block(kThreads);
  if (src_f64 && dst_f64)
    box_kernel<double, double><<<grid, block, 0, s>>>(items, terms, ptrs);
  else if (!src_f64 && !dst_f64)
    box_kernel<float, float><<<grid, block, 0, s>>>(items, terms, ptrs);
  else
    return (int)cudaErrorInvalidValue;
  return (int)cudaGetLastError();
}

}  // namespace sym
