// Block movement kernel: every permute / fuse / split / matrix-form gather /
// scatter of the library is a set of strided boxes, each destination element
// being a short sum of coefficient x source element (one term for U(1) and
// for pure re-indexing; the recoupling sum of Ch. 6, Eq. permsu2, for SU(2)).
//
// One CTA handles one BoxItem (a chunk of at most kBoxChunk elements of one
// box).  Threads walk the chunk in the box's row-major order, which the
// planner chooses so that the source's fastest dimension is the box's last
// dimension (coalesced reads).  Memory-bound: bytes = read src + write dst.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace sym {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxSmemTerms = 64;

struct TermF {
  int64_t off;
  int64_t ld;
};

template <typename TS, int MODE>
__global__ void __launch_bounds__(kThreads) box_kernel(const BoxItem* __restrict__ items,
                                                       const Term* __restrict__ terms,
                                                       const BoxPtrs ptrs) {
  __shared__ BoxItem it;
  __shared__ TermF toff[kMaxSmemTerms];
  __shared__ double tcoef[kMaxSmemTerms];
  if (threadIdx.x == 0) it = items[blockIdx.x];
  __syncthreads();
  const int nterm = it.nterm;
  for (int i = threadIdx.x; i < nterm && i < kMaxSmemTerms; i += blockDim.x) {
    Term t = terms[it.term0 + i];
    toff[i] = TermF{t.off, t.ld};
    tcoef[i] = t.coef;
  }
  __syncthreads();
  const int ndim = it.ndim;
  const TS* __restrict__ src = static_cast<const TS*>(ptrs.src[it.sel & 3]);
  void* dst0 = ptrs.dst[(it.sel >> 4) & 3][0];
  void* dst1 = ptrs.dst[(it.sel >> 4) & 3][1];
  for (int e = threadIdx.x; e < it.count; e += blockDim.x) {
    int rem = it.start + e;
    int sa = 0, sb = 0, da = 0, db = 0;
#pragma unroll
    for (int d = kMaxDim - 1; d >= 0; --d) {
      if (d < ndim) {
        int n = it.dims[d];
        int q = rem / n;
        int t = rem - q * n;
        rem = q;
        sa += t * it.sa[d];
        sb += t * it.sb[d];
        da += t * it.da[d];
        db += t * it.db[d];
      }
    }
    if constexpr (sizeof(TS) == 8) {
      double acc = 0.0;
      for (int i = 0; i < nterm; ++i) {
        const int64_t off = i < kMaxSmemTerms ? toff[i].off + toff[i].ld * sa : terms[it.term0 + i].off + terms[it.term0 + i].ld * sa;
        const double c = i < kMaxSmemTerms ? tcoef[i] : terms[it.term0 + i].coef;
        acc = fma(c, (double)src[off + sb], acc);
      }
      if constexpr (MODE == BOX_LINEAR_F64) {
        static_cast<double*>(dst0)[it.dst_off + (int64_t)it.dst_ld * da + db] = acc;
      } else if constexpr (MODE == BOX_LINEAR_F32) {
        static_cast<float*>(dst0)[it.dst_off + (int64_t)it.dst_ld * da + db] = (float)acc;
      }
    } else {
      float acc = 0.0f;
      for (int i = 0; i < nterm; ++i) {
        const int64_t off = i < kMaxSmemTerms ? toff[i].off + toff[i].ld * sa : terms[it.term0 + i].off + terms[it.term0 + i].ld * sa;
        const float c = (float)(i < kMaxSmemTerms ? tcoef[i] : terms[it.term0 + i].coef);
        acc = fmaf(c, (float)src[off + sb], acc);
      }
      if constexpr (MODE == BOX_LINEAR_F32) {
        static_cast<float*>(dst0)[it.dst_off + (int64_t)it.dst_ld * da + db] = acc;
      } else if constexpr (MODE == BOX_LINEAR_F64) {
        static_cast<double*>(dst0)[it.dst_off + (int64_t)it.dst_ld * da + db] = (double)acc;
      } else {
        // split-BF16: hi = bf16(v), lo = bf16(v - hi); tiled, 128B-swizzled image
        const int row = it.row0 + da;
        const int col = it.col0 + db;
        const int64_t off = it.dst_off + ((int64_t)(row >> 7) * it.dst_ld + (col >> 6)) * 8192 +
                            (row & 127) * 64 + ((((col >> 3) & 7) ^ (row & 7)) << 3) + (col & 7);
        const __nv_bfloat16 hi = __float2bfloat16_rn(acc);
        const __nv_bfloat16 lo = __float2bfloat16_rn(acc - __bfloat162float(hi));
        static_cast<__nv_bfloat16*>(dst0)[off] = hi;
        static_cast<__nv_bfloat16*>(dst1)[off] = lo;
      }
    }
  }
}

}  // namespace

int launch_box(int mode, bool src_f64, const BoxItem* items, int nitems, const Term* terms, const BoxPtrs& ptrs,
               void* stream) {
  if (nitems <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid(nitems), block(kThreads);
  if (src_f64) {
    if (mode == BOX_LINEAR_F64)
      box_kernel<double, BOX_LINEAR_F64><<<grid, block, 0, s>>>(items, terms, ptrs);
    else if (mode == BOX_LINEAR_F32)
      box_kernel<double, BOX_LINEAR_F32><<<grid, block, 0, s>>>(items, terms, ptrs);
    else
      return (int)cudaErrorInvalidValue;
  } else {
    if (mode == BOX_LINEAR_F32)
      box_kernel<float, BOX_LINEAR_F32><<<grid, block, 0, s>>>(items, terms, ptrs);
    else if (mode == BOX_LINEAR_F64)
      box_kernel<float, BOX_LINEAR_F64><<<grid, block, 0, s>>>(items, terms, ptrs);
    else
      box_kernel<float, BOX_IMAGE_BF16X2><<<grid, block, 0, s>>>(items, terms, ptrs);
  }
  return (int)cudaGetLastError();
}

}  // namespace sym
