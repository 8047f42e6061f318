// Direct contraction of sectors with a tiny matrix on one side.
//
// Blockwise matrix multiply of Ch. 5, Eq. blockmult, T_j = M_j N_j, for the
// sectors j whose N_j is at most kMaxDirect x kMaxDirect (an MPO or a
// physical leg on the contracted side).  Moving such a sector into matrix
// form and back would cost two extra passes over the large operand for a
// GEMM that is itself a pure stream, so the product is taken on the blocks:
// a work item is one row group of the sector (the blocks of the large
// operand that share the charges of their free legs), its box the free legs,
// its source and destination columns the positions of the contracted and of
// the other operand's free legs inside those blocks.
//
//   apply  C_d[t] = sum_s N(s, d) A_s[t]   (forward, and dA = dC N^T)
//   outer  dN(s, d) += sum_t A_s[t] dC_d[t] (dB = A^T dC), reduced across the
//          warp with butterfly shuffles and added into the zero-filled
//          gradient blocks with atomics
//
// Persistent and warp-independent: a warp copies one 128-byte descriptor into
// its shared-memory slot, stages the item's coefficients and column pointers
// in registers, and streams the box with coalesced loads along its last dim.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"
#include "pdl.h"

namespace sym {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kH = 4;   // positions in flight per lane (apply)
constexpr int kHo = 2;  // (outer: twice the columns per position)

template <typename T>
__device__ __forceinline__ T coef_of(const Term& t);
template <>
__device__ __forceinline__ float coef_of<float>(const Term& t) { return t.coef_f; }
template <>
__device__ __forceinline__ double coef_of<double>(const Term& t) { return t.coef; }

template <typename T>
__device__ __forceinline__ const T* src_ptr(const BoxPtrs& p, int slot) {
  return static_cast<const T*>(slot == 0 ? p.src[0] : slot == 1 ? p.src[1] : slot == 2 ? p.src[2] : p.src[3]);
}

template <typename T>
__device__ __forceinline__ T* dst_ptr(const BoxPtrs& p, int slot) {
  return static_cast<T*>(slot == DST_OUT ? p.dst[DST_OUT] : slot == DST_DA ? p.dst[DST_DA] : p.dst[DST_DB]);
}

// box index of position e (last dim fastest); floor(r / n) = umulhi(2r, mag) >> shf
struct DirectShape {
  int n[kDirectDims], shf[kDirectDims];
  uint32_t mag[kDirectDims];
  int sa[kDirectDims], sb[kDirectDims], da[kDirectDims], db[kDirectDims];
  __device__ __forceinline__ explicit DirectShape(const DirectItem& it) {
#pragma unroll
    for (int d = 0; d < kDirectDims; ++d) {
      n[d] = it.dims[d];
      mag[d] = it.mag[d];
      shf[d] = (it.shf >> (8 * d)) & 0xff;
      sa[d] = it.sa[d];
      sb[d] = it.sb[d];
      da[d] = it.da[d];
      db[d] = it.db[d];
    }
  }
  // source (ld multiplier a, offset b) and destination (c, e) parts of position p
  __device__ __forceinline__ void at(int p, int& a, int& b, int& c, int& e) const {
    int t[kDirectDims];
    int rem = p;
#pragma unroll
    for (int d = kDirectDims - 1; d > 0; --d) {
      const int q = (int)(__umulhi((uint32_t)rem << 1, mag[d]) >> shf[d]);
      t[d] = rem - q * n[d];
      rem = q;
    }
    t[0] = rem;
    a = b = c = e = 0;
#pragma unroll
    for (int d = 0; d < kDirectDims; ++d) {
      a += t[d] * sa[d];
      b += t[d] * sb[d];
      c += t[d] * da[d];
      e += t[d] * db[d];
    }
  }
};

template <typename T>
__device__ __forceinline__ void apply_item(const DirectItem& it, const Term* __restrict__ terms, const BoxPtrs& ptrs,
                                           int lane) {
  const int ns = it.ns, nd = it.nd;
  const T* __restrict__ src = src_ptr<T>(ptrs, it.slots & 3);
  const T* __restrict__ ksrc = src_ptr<T>(ptrs, (it.slots >> 2) & 3);
  T* __restrict__ dst = dst_ptr<T>(ptrs, (it.slots >> 4) & 7);
  const T* sp[kMaxDirect];
  T* dp[kMaxDirect];
  int sl[kMaxDirect], dl[kMaxDirect];
  T cf[kMaxDirect][kMaxDirect];
#pragma unroll
  for (int s = 0; s < kMaxDirect; ++s) {
    const bool on = s < ns;
    const Term t = terms[it.ts + (on ? s : 0)];
    sp[s] = src + t.off;
    sl[s] = on ? (int)t.ld : 0;
  }
#pragma unroll
  for (int d = 0; d < kMaxDirect; ++d) {
    const bool on = d < nd;
    const Term t = terms[it.td + (on ? d : 0)];
    dp[d] = dst + t.off;
    dl[d] = on ? (int)t.ld : 0;
  }
#pragma unroll
  for (int d = 0; d < kMaxDirect; ++d)
#pragma unroll
    for (int s = 0; s < kMaxDirect; ++s) {
      cf[d][s] = T(0);
      if (d < nd && s < ns) {
        const Term t = terms[it.tk + d * it.kd + s * it.ks];
        const T c = coef_of<T>(t);
        if (c != T(0)) cf[d][s] = c * __ldg(ksrc + t.off);
      }
    }
  const DirectShape sh(it);
  const int last = it.start + it.count - 1;
#pragma unroll 1
  for (int u = it.start + lane; u <= last; u += 32 * kH) {
    int c[kH], e[kH];
    T v[kH][kMaxDirect];
#pragma unroll
    for (int h = 0; h < kH; ++h) {
      int a, b;
      sh.at(min(u + 32 * h, last), a, b, c[h], e[h]);
#pragma unroll
      for (int s = 0; s < kMaxDirect; ++s) v[h][s] = s < ns ? __ldg(sp[s] + (int64_t)sl[s] * a + b) : T(0);
    }
#pragma unroll
    for (int h = 0; h < kH; ++h) {
      if (u + 32 * h > last) break;
#pragma unroll
      for (int d = 0; d < kMaxDirect; ++d) {
        if (d >= nd) break;
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < kMaxDirect; ++s) acc = fma(cf[d][s], v[h][s], acc);
        dp[d][(int64_t)dl[d] * c[h] + e[h]] = acc;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void outer_item(const DirectItem& it, const Term* __restrict__ terms, const BoxPtrs& ptrs,
                                           int lane) {
  const int ns = it.ns, nd = it.nd;
  const T* __restrict__ src = src_ptr<T>(ptrs, it.slots & 3);
  const T* __restrict__ src2 = src_ptr<T>(ptrs, (it.slots >> 2) & 3);
  T* __restrict__ dst = dst_ptr<T>(ptrs, (it.slots >> 4) & 7);
  const T* sp[kMaxDirect];
  const T* qp[kMaxDirect];
  int sl[kMaxDirect], ql[kMaxDirect];
#pragma unroll
  for (int s = 0; s < kMaxDirect; ++s) {
    const bool on = s < ns;
    const Term t = terms[it.ts + (on ? s : 0)];
    sp[s] = src + t.off;
    sl[s] = on ? (int)t.ld : 0;
  }
#pragma unroll
  for (int d = 0; d < kMaxDirect; ++d) {
    const bool on = d < nd;
    const Term t = terms[it.td + (on ? d : 0)];
    qp[d] = src2 + t.off;
    ql[d] = on ? (int)t.ld : 0;
  }
  T acc[kMaxDirect][kMaxDirect];
#pragma unroll
  for (int s = 0; s < kMaxDirect; ++s)
#pragma unroll
    for (int d = 0; d < kMaxDirect; ++d) acc[s][d] = T(0);
  const DirectShape sh(it);
  const int last = it.start + it.count - 1;
#pragma unroll 1
  for (int u = it.start + lane; u <= last; u += 32 * kHo) {
    T va[kHo][kMaxDirect], vq[kHo][kMaxDirect];
#pragma unroll
    for (int h = 0; h < kHo; ++h) {
      const bool ok = u + 32 * h <= last;
      int a, b, c, e;
      sh.at(min(u + 32 * h, last), a, b, c, e);
#pragma unroll
      for (int s = 0; s < kMaxDirect; ++s) va[h][s] = (ok && s < ns) ? __ldg(sp[s] + (int64_t)sl[s] * a + b) : T(0);
#pragma unroll
      for (int d = 0; d < kMaxDirect; ++d) vq[h][d] = (ok && d < nd) ? __ldg(qp[d] + (int64_t)ql[d] * c + e) : T(0);
    }
#pragma unroll
    for (int h = 0; h < kHo; ++h)
#pragma unroll
      for (int s = 0; s < kMaxDirect; ++s)
#pragma unroll
        for (int d = 0; d < kMaxDirect; ++d) acc[s][d] = fma(va[h][s], vq[h][d], acc[s][d]);
  }
  // butterfly: every lane ends with the warp's sums
#pragma unroll
  for (int s = 0; s < kMaxDirect; ++s)
#pragma unroll
    for (int d = 0; d < kMaxDirect; ++d)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[s][d] += __shfl_xor_sync(0xffffffffu, acc[s][d], o);
  // lane s * kMaxDirect + d adds out(s, d)
  const int s0 = lane / kMaxDirect, d0 = lane % kMaxDirect;
  if (lane < kMaxDirect * kMaxDirect && s0 < ns && d0 < nd) {
    T v = T(0);
#pragma unroll
    for (int s = 0; s < kMaxDirect; ++s)
#pragma unroll
      for (int d = 0; d < kMaxDirect; ++d)
        if (s == s0 && d == d0) v = acc[s][d];
    const Term t = terms[it.tk + d0 * it.kd + s0 * it.ks];
    const T c = coef_of<T>(t);
    if (c != T(0)) atomicAdd(dst + t.off, c * v);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) direct_kernel(const DirectItem* __restrict__ items, int nitems,
                                                          const Term* __restrict__ terms, BoxPtrs ptrs) {
  constexpr int kWords = sizeof(DirectItem) / 4;
  static_assert(kWords <= 32, "one descriptor word per lane");
  __shared__ uint32_t desc[kWarps][kWords];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pdl_wait();
  pdl_launch_dependents();
  for (int w = blockIdx.x * kWarps + warp; w < nitems; w += gridDim.x * kWarps) {
    __syncwarp();
    if (lane < kWords) desc[warp][lane] = reinterpret_cast<const uint32_t*>(items + w)[lane];
    __syncwarp();
    const DirectItem& it = *reinterpret_cast<const DirectItem*>(desc[warp]);
    if (it.op == kDirectApply)
      apply_item<T>(it, terms, ptrs, lane);
    else
      outer_item<T>(it, terms, ptrs, lane);
  }
}

template <typename T>
int ctas_per_sm() {
  static const int n = [] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, direct_kernel<T>, kThreads, 0) != cudaSuccess || v < 1)
      v = 1;
    return v;
  }();
  return n;
}

template <typename T>
int launch_t(const DirectItem* items, int nitems, const Term* terms, const BoxPtrs& ptrs, cudaStream_t s) {
  const int ctas = std::min((nitems + kWarps - 1) / kWarps, tc_num_sms() * ctas_per_sm<T>());
  return (int)launch_pdl(direct_kernel<T>, dim3(ctas), dim3(kThreads), 0, s, items, nitems, terms, ptrs);
}

}  // namespace

int launch_direct(bool f64, const DirectItem* items, int nitems, const Term* terms, const BoxPtrs& ptrs,
                  void* stream) {
  if (nitems <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return f64 ? launch_t<double>(items, nitems, terms, ptrs, s) : launch_t<float>(items, nitems, terms, ptrs, s);
}

}  // namespace sym
