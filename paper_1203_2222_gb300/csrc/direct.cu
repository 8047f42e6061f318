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
// Persistent and warp-independent: a warp copies one 512-byte descriptor
// (columns inline) into its shared-memory slot while the previous item runs,
// stages the item's coefficients and column pointers in registers, and
// streams the box with coalesced loads along its last dim.
// Apply and outer items run as separate launches of their own kernels (every
// item of a launch has the same kind).
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"
#include "pdl.h"

namespace sym {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
// Loads are staged by cp.async into a per-lane slice of shared memory, two
// stages deep, so that a lane keeps 2 * kH(T) positions x kMaxDirect columns
// in flight (2 * 8 KB per warp) without holding them in registers; each lane
// reads back only what it copied itself, so no barrier is needed.
template <typename T>
constexpr int kH = 32 / (int)sizeof(T);  // apply: positions per lane per stage (8 fp32, 4 fp64)
template <typename T>
constexpr int kHo = kH<T> / 2;           // outer: (twice the columns per position)
constexpr int kStageBytes = 32 * 32 * kMaxDirect;  // one stage of one warp: 32 lanes x 8 fp32 x 4 columns

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ const T* src_ptr(const BoxPtrs& p, int slot) {
  return static_cast<const T*>(slot == 0 ? p.src[0] : slot == 1 ? p.src[1] : slot == 2 ? p.src[2] : p.src[3]);
}

template <typename T>
__device__ __forceinline__ T* dst_ptr(const BoxPtrs& p, int slot) {
  return static_cast<T*>(slot == DST_OUT ? p.dst[DST_OUT] : slot == DST_DA ? p.dst[DST_DA] : p.dst[DST_DB]);
}

// Box index of position p (last dim fastest): floor(r / n) = umulhi(2r, mag) >> shf.
// ND = the item's number of dims (1..3); one dim needs no division.
template <int ND>
struct DirectShape {
  int n[ND], shf[ND];
  uint32_t mag[ND];
  __device__ __forceinline__ explicit DirectShape(const DirectItem& it) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      n[d] = it.dims[d];
      mag[d] = it.mag[d];
      shf[d] = (it.shf >> (8 * d)) & 0xff;
    }
  }
  __device__ __forceinline__ void index(int p, int (&t)[ND]) const {
    int rem = p;
#pragma unroll
    for (int d = ND - 1; d > 0; --d) {
      const int q = (int)(__umulhi((uint32_t)rem << 1, mag[d]) >> shf[d]);
      t[d] = rem - q * n[d];
      rem = q;
    }
    t[0] = rem;
  }
};

// Columns of one side of an item: column c at box index t is base[c][<t, str[c]>]
// (the relative offset stays below 2^31 -- host check -- so it is formed in 32 bits).
template <typename P, int NC, int ND>
struct Cols {
  P base[NC];
  int str[NC][ND];
  __device__ __forceinline__ void load(P slot, const DirectCol* cols, int n) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const bool on = c < n;
      base[c] = slot + cols[on ? c : 0].off;
#pragma unroll
      for (int d = 0; d < ND; ++d) str[c][d] = on ? cols[c].str[d] : 0;
    }
  }
  __device__ __forceinline__ int off(int c, const int (&t)[ND]) const {
    int o = 0;
#pragma unroll
    for (int d = 0; d < ND; ++d) o += t[d] * str[c][d];
    return o;
  }
};

// apply: NS source and NQ destination columns (exact counts when the item has
// them, else upper bounds with the actual counts ns <= NS, nq <= NQ); the
// coefficient values are in this warp's cf[d * kMaxDirect + s]
template <typename T, int ND, int NS, int NQ>
__device__ __forceinline__ void apply_item(const DirectItem& it, const T* __restrict__ cfv, const BoxPtrs& ptrs,
                                           int lane, T* __restrict__ stage) {
  const int ns = it.ns, nq = it.nd;
  Cols<const T*, NS, ND> S;
  Cols<T*, NQ, ND> Q;
  S.load(src_ptr<T>(ptrs, it.slots & 3), it.src, ns);
  Q.load(dst_ptr<T>(ptrs, (it.slots >> 4) & 7), it.dst, nq);
  T cf[NQ][NS];
#pragma unroll
  for (int d = 0; d < NQ; ++d)
#pragma unroll
    for (int c = 0; c < NS; ++c) cf[d][c] = (d < nq && c < ns) ? cfv[d * kMaxDirect + c] : T(0);
  const DirectShape<ND> sh(it);
  const int last = it.start + it.count - 1;
  constexpr int H = kH<T>;
  constexpr int SLOT = H * NS * 32;  // one stage: [H][NS][32], this lane's values at [..][..][lane]
  auto issue = [&](int u, T* buf) {
#pragma unroll
    for (int h = 0; h < H; ++h) {
      int t[ND];
      sh.index(min(u + 32 * h, last), t);
#pragma unroll
      for (int c = 0; c < NS; ++c)
        if (c < ns) cp_async(buf + (h * NS + c) * 32 + lane, S.base[c] + S.off(c, t), sizeof(T));
    }
    cp_commit();
  };
  const int step = 32 * H;
  int u = it.start + lane;
  if (u <= last) issue(u, stage);
  for (int k = 0; u <= last; u += step, ++k) {
    T* cur = stage + (k & 1) * SLOT;
    if (u + step <= last) {
      issue(u + step, stage + ((k + 1) & 1) * SLOT);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      if (u + 32 * h > last) break;
      int t[ND];
      sh.index(u + 32 * h, t);
      T v[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) v[c] = c < ns ? cur[(h * NS + c) * 32 + lane] : T(0);
#pragma unroll
      for (int d = 0; d < NQ; ++d) {
        if (d >= nq) break;
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < NS; ++c) acc = fma(cf[d][c], v[c], acc);
        Q.base[d][Q.off(d, t)] = acc;
      }
    }
  }
}

// outer: out(s, d) = sum_t A_s[t] dC_d[t] over the item's positions, scaled
// by kc and added into the destination at koff
template <typename T, int ND, int NS, int NQ>
__device__ __forceinline__ void outer_item(const DirectItem& it, const BoxPtrs& ptrs, int lane,
                                           T* __restrict__ stage) {
  const int ns = it.ns, nq = it.nd;
  T* __restrict__ dst = dst_ptr<T>(ptrs, (it.slots >> 4) & 7);
  Cols<const T*, NS, ND> S;
  Cols<const T*, NQ, ND> Q;
  S.load(src_ptr<T>(ptrs, it.slots & 3), it.src, ns);
  Q.load(src_ptr<T>(ptrs, (it.slots >> 2) & 3), it.dst, nq);
  T acc[NS][NQ];
#pragma unroll
  for (int c = 0; c < NS; ++c)
#pragma unroll
    for (int d = 0; d < NQ; ++d) acc[c][d] = T(0);
  const DirectShape<ND> sh(it);
  const int last = it.start + it.count - 1;
  constexpr int H = kHo<T>;
  constexpr int W = NS + NQ;          // values per position
  constexpr int SLOT = H * W * 32;    // one stage: [H][W][32]
  auto issue = [&](int u, T* buf) {
#pragma unroll
    for (int h = 0; h < H; ++h) {
      int t[ND];
      sh.index(min(u + 32 * h, last), t);
#pragma unroll
      for (int c = 0; c < NS; ++c)
        if (c < ns) cp_async(buf + (h * W + c) * 32 + lane, S.base[c] + S.off(c, t), sizeof(T));
#pragma unroll
      for (int d = 0; d < NQ; ++d)
        if (d < nq) cp_async(buf + (h * W + NS + d) * 32 + lane, Q.base[d] + Q.off(d, t), sizeof(T));
    }
    cp_commit();
  };
  const int step = 32 * H;
  int u = it.start + lane;
  if (u <= last) issue(u, stage);
  for (int k = 0; u <= last; u += step, ++k) {
    T* cur = stage + (k & 1) * SLOT;
    if (u + step <= last) {
      issue(u + step, stage + ((k + 1) & 1) * SLOT);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      if (u + 32 * h > last) break;
      T va[NS], vq[NQ];
#pragma unroll
      for (int c = 0; c < NS; ++c) va[c] = c < ns ? cur[(h * W + c) * 32 + lane] : T(0);
#pragma unroll
      for (int d = 0; d < NQ; ++d) vq[d] = d < nq ? cur[(h * W + NS + d) * 32 + lane] : T(0);
#pragma unroll
      for (int c = 0; c < NS; ++c)
#pragma unroll
        for (int d = 0; d < NQ; ++d) acc[c][d] = fma(va[c], vq[d], acc[c][d]);
    }
  }
  // butterfly: every lane ends with the warp's sums
#pragma unroll
  for (int c = 0; c < NS; ++c)
#pragma unroll
    for (int d = 0; d < NQ; ++d)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c][d] += __shfl_xor_sync(0xffffffffu, acc[c][d], o);
  // lane c * NQ + d adds out(c, d)
  const int c0 = lane / NQ, d0 = lane % NQ;
  if (lane < NS * NQ && c0 < ns && d0 < nq) {
    T v = T(0);
#pragma unroll
    for (int c = 0; c < NS; ++c)
#pragma unroll
      for (int d = 0; d < NQ; ++d)
        if (c == c0 && d == d0) v = acc[c][d];
    const int e = d0 * kMaxDirect + c0;
    const double k = it.kc[e];
    if (k != 0.0) atomicAdd(dst + it.koff[e], T(k) * v);
  }
}

// the item's column counts pick an exact variant (the MPO and physical legs
// of a tensor network give 1 or 4 columns per side), else the bounded one
template <typename T, int kOp, int ND>
__device__ __forceinline__ void run_item(const DirectItem& it, const T* __restrict__ cfv, const BoxPtrs& ptrs,
                                         int lane, T* __restrict__ stage) {
  const int key = ND == 3 ? 0 : it.ns * 8 + it.nd;  // three-dim boxes take the bounded variant only
  if (kOp == kDirectApply) {
    if (key == 4 * 8 + 4) apply_item<T, ND, 4, 4>(it, cfv, ptrs, lane, stage);
    else if (key == 1 * 8 + 1) apply_item<T, ND, 1, 1>(it, cfv, ptrs, lane, stage);
    else if (key == 1 * 8 + 4) apply_item<T, ND, 1, 4>(it, cfv, ptrs, lane, stage);
    else if (key == 4 * 8 + 1) apply_item<T, ND, 4, 1>(it, cfv, ptrs, lane, stage);
    else apply_item<T, ND, kMaxDirect, kMaxDirect>(it, cfv, ptrs, lane, stage);
  } else {
    if (key == 4 * 8 + 4) outer_item<T, ND, 4, 4>(it, ptrs, lane, stage);
    else if (key == 1 * 8 + 1) outer_item<T, ND, 1, 1>(it, ptrs, lane, stage);
    else if (key == 1 * 8 + 4) outer_item<T, ND, 1, 4>(it, ptrs, lane, stage);
    else if (key == 4 * 8 + 1) outer_item<T, ND, 4, 1>(it, ptrs, lane, stage);
    else outer_item<T, ND, kMaxDirect, kMaxDirect>(it, ptrs, lane, stage);
  }
}

// One kernel per item kind, so that each gets the registers of its own loop.
// A warp keeps the next item's descriptor in flight (one 16-byte load per
// lane) while it runs the current one, so an item's set-up costs one round
// trip: the apply coefficients, loaded by one lane each.
template <typename T, int kOp>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2)
    direct_kernel(const DirectItem* __restrict__ items, int nitems, BoxPtrs ptrs) {
  static_assert(sizeof(DirectItem) == 32 * sizeof(int4), "one 16-byte descriptor word per lane");
  __shared__ __align__(16) DirectItem desc[kWarps];
  __shared__ T cfs[kWarps][kMaxDirect * kMaxDirect];
  extern __shared__ __align__(16) unsigned char dyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* stage = reinterpret_cast<T*>(dyn + (size_t)warp * 2 * kStageBytes);
  const int stride = gridDim.x * kWarps;
  int w = blockIdx.x * kWarps + warp;
  int4 next = make_int4(0, 0, 0, 0);
  if (w < nitems) next = __ldg(reinterpret_cast<const int4*>(items + w) + lane);
  pdl_wait();
  pdl_launch_dependents();
  for (; w < nitems; w += stride) {
    __syncwarp();
    reinterpret_cast<int4*>(desc + warp)[lane] = next;
    __syncwarp();
    if (w + stride < nitems) next = __ldg(reinterpret_cast<const int4*>(items + w + stride) + lane);
    const DirectItem& it = desc[warp];
    if (kOp == kDirectApply) {  // coefficient values, one lane each
      const T* __restrict__ ksrc = src_ptr<T>(ptrs, (it.slots >> 2) & 3);
      if (lane < kMaxDirect * kMaxDirect) {
        const double k = it.kc[lane];
        cfs[warp][lane] = k != 0.0 ? T(k) * __ldg(ksrc + it.koff[lane]) : T(0);
      }
      __syncwarp();
    }
    if (it.ndim == 1)
      run_item<T, kOp, 1>(it, cfs[warp], ptrs, lane, stage);
    else if (it.ndim == 2)
      run_item<T, kOp, 2>(it, cfs[warp], ptrs, lane, stage);
    else
      run_item<T, kOp, 3>(it, cfs[warp], ptrs, lane, stage);
  }
}

constexpr int kDynSmem = kWarps * 2 * kStageBytes;  // 64 KB: two stages per warp

template <typename T, int kOp>
int ctas_per_sm() {
  static const int n = [] {
    int v = 0;
    cudaFuncSetAttribute(direct_kernel<T, kOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, direct_kernel<T, kOp>, kThreads, kDynSmem) != cudaSuccess ||
        v < 1)
      v = 1;
    return v;
  }();
  return n;
}

template <typename T, int kOp>
int launch_op(const DirectItem* items, int nitems, const BoxPtrs& ptrs, cudaStream_t s) {
  if (nitems <= 0) return 0;
  const int ctas = std::min((nitems + kWarps - 1) / kWarps, tc_num_sms() * ctas_per_sm<T, kOp>());
  return (int)launch_pdl(direct_kernel<T, kOp>, dim3(ctas), dim3(kThreads), kDynSmem, s, items, nitems, ptrs);
}

}  // namespace

int launch_direct(bool f64, int op, const DirectItem* items, int nitems, const BoxPtrs& ptrs, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (op == kDirectApply)
    return f64 ? launch_op<double, kDirectApply>(items, nitems, ptrs, s)
               : launch_op<float, kDirectApply>(items, nitems, ptrs, s);
  return f64 ? launch_op<double, kDirectOuter>(items, nitems, ptrs, s)
             : launch_op<float, kDirectOuter>(items, nitems, ptrs, s);
}

}  // namespace sym
