// Block movement kernel: every permute / fuse / split / matrix-form gather /
// scatter of the library is a set of strided boxes, each destination element
// being a short sum of coefficient x source element (one term for U(1) and
// for pure re-indexing; the recoupling sum of Ch. 6, Eq. permsu2, for SU(2)).
//
// One CTA handles one BoxItem (a chunk of one box).  The planner orders each
// box so that its last dimension is the source's fastest one; the CTA walks
// the chunk row by row (a row = the last dimension): with rows of 32 or more
// elements one warp takes a row and its lanes run along it (coalesced reads,
// one index decomposition per row), shorter rows go thread per element.
// Memory-bound: bytes = source read + destination written.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace sym {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxSmemTerms = 64;
constexpr int kItemWords = (int)(sizeof(BoxItem) / 4);
static_assert(sizeof(BoxItem) % 4 == 0, "BoxItem must be a whole number of words");

template <typename TS, typename TD>
struct BoxCtx {
  const BoxItem* it;
  const Term* terms;
  const int64_t* toff;
  const int64_t* tld;
  const double* tcoef;
  const TS* src;
  void* dst0;
  void* dst1;
  bool image;

  __device__ __forceinline__ void element(int sa, int sb, int da, int db) const {
    const int nterm = it->nterm;
    TD acc = TD(0);
    for (int i = 0; i < nterm; ++i) {
      int64_t off;
      double c;
      if (i < kMaxSmemTerms) {
        off = toff[i] + tld[i] * sa;
        c = tcoef[i];
      } else {
        const Term t = terms[it->term0 + i];
        off = t.off + t.ld * sa;
        c = t.coef;
      }
      acc += TD(c) * TD(src[off + sb]);
    }
    if (!image) {
      static_cast<TD*>(dst0)[it->dst_off + (int64_t)it->dst_ld * da + db] = acc;
    } else {
      // split-BF16: hi = bf16(v), lo = bf16(v - hi); tiled, 128B-swizzled image
      const float v = (float)acc;
      const int row = it->row0 + da;
      const int col = it->col0 + db;
      const int64_t off = it->dst_off + ((int64_t)(row >> 7) * it->dst_ld + (col >> 6)) * 8192 +
                          (row & 127) * 64 + ((((col >> 3) & 7) ^ (row & 7)) << 3) + (col & 7);
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      static_cast<__nv_bfloat16*>(dst0)[off] = hi;
      static_cast<__nv_bfloat16*>(dst1)[off] = lo;
    }
  }
};

template <typename TS, typename TD>
__global__ void __launch_bounds__(kThreads) box_kernel(const BoxItem* __restrict__ items,
                                                       const Term* __restrict__ terms, const BoxPtrs ptrs) {
  __shared__ int32_t raw[kItemWords];
  __shared__ int64_t toff[kMaxSmemTerms], tld[kMaxSmemTerms];
  __shared__ double tcoef[kMaxSmemTerms];
  const int32_t* g = reinterpret_cast<const int32_t*>(items + blockIdx.x);
  for (int i = threadIdx.x; i < kItemWords; i += blockDim.x) raw[i] = g[i];
  __syncthreads();
  const BoxItem& it = *reinterpret_cast<const BoxItem*>(raw);
  for (int i = threadIdx.x; i < it.nterm && i < kMaxSmemTerms; i += blockDim.x) {
    const Term t = terms[it.term0 + i];
    toff[i] = t.off;
    tld[i] = t.ld;
    tcoef[i] = t.coef;
  }
  __syncthreads();
  const int dslot = (it.sel >> 4) & 7;
  BoxCtx<TS, TD> ctx{&it, terms, toff, tld, tcoef, static_cast<const TS*>(ptrs.src[it.sel & 3]),
                     ptrs.dst[dslot][0], ptrs.dst[dslot][1], (it.sel & kSelImage) != 0};
  const int nd = it.ndim;
  const int L = it.dims[nd - 1];
  const int s_a = it.sa[nd - 1], s_b = it.sb[nd - 1], d_a = it.da[nd - 1], d_b = it.db[nd - 1];
  const int e0 = it.start, e1 = it.start + it.count;
  if (L >= 32) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int r0 = e0 / L, r1 = (e1 - 1) / L;
    for (int r = r0 + warp; r <= r1; r += nwarps) {
      int rem = r, sa = 0, sb = 0, da = 0, db = 0;
#pragma unroll
      for (int d = kMaxDim - 2; d >= 0; --d) {
        if (d < nd - 1) {
          const int n = it.dims[d];
          const int q = rem / n;
          const int t = rem - q * n;
          rem = q;
          sa += t * it.sa[d];
          sb += t * it.sb[d];
          da += t * it.da[d];
          db += t * it.db[d];
        }
      }
      const int i0 = max(e0 - r * L, 0), i1 = min(e1 - r * L, L);
      for (int i = i0 + lane; i < i1; i += 32) ctx.element(sa + i * s_a, sb + i * s_b, da + i * d_a, db + i * d_b);
    }
  } else {
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int rem = e, sa = 0, sb = 0, da = 0, db = 0;
#pragma unroll
      for (int d = kMaxDim - 1; d >= 0; --d) {
        if (d < nd) {
          const int n = it.dims[d];
          const int q = rem / n;
          const int t = rem - q * n;
          rem = q;
          sa += t * it.sa[d];
          sb += t * it.sb[d];
          da += t * it.da[d];
          db += t * it.db[d];
        }
      }
      ctx.element(sa, sb, da, db);
    }
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
