// Block movement kernel: every permute / fuse / split / matrix-form gather /
// scatter of the library is a set of strided boxes, each destination element
// being a short sum of coefficient x source element (one term for U(1) and
// for pure re-indexing; the recoupling sum of Ch. 6, Eq. permsu2, for SU(2)).
//
// The kernel is persistent and its warps are independent: warp g of the grid
// takes items g, g + W, g + 2W, ... (W warps in all), keeps the current
// descriptor in its own slice of shared memory, fetches the next one into
// registers while it works, and never waits on the rest of its CTA.
//  - A linear item is at most 512 elements of one box, 16 per lane; lane l
//    takes elements start + l + 32u, so consecutive lanes read consecutive
//    source elements (the planner makes the box's last dim the source's
//    fastest).  The multi-index of an element is split off by multiply-high
//    division (magic numbers from the planner) in registers, with the number
//    of dims a template parameter; all 16 loads are issued before any store.
//  - A flat item (at most one term, 32-bit spans) addresses both sides with
//    a single dot product each; the general form (recoupling sums, offsets
//    beyond 32 bits) keeps the two-part source and destination offsets.
//  - A tile item is one 32 x 32 tile of the box's last two dims at one outer
//    index: the warp reads it along the source-contiguous dim into its own
//    shared-memory tile and writes it along the destination-contiguous dim.
// Memory-bound: bytes = source read + destination written.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "pdl.h"

namespace sym {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kBatch = kBoxChunk / 32;  // elements per lane of a linear item
constexpr int kItemWords = (int)(sizeof(BoxItem) / 8);
static_assert(sizeof(BoxItem) % 8 == 0, "BoxItem must be a whole number of 8-byte words");
static_assert(kItemWords <= 32, "a warp loads a descriptor with one word per lane");

// coefficient in the data type: FP32 kernels read the planner's FP32 copy
// and so issue no FP64 instruction (FP64 is a low-rate pipe)
template <typename TD>
__device__ __forceinline__ TD coef(double c, float cf);
template <>
__device__ __forceinline__ double coef<double>(double c, float) { return c; }
template <>
__device__ __forceinline__ float coef<float>(double, float cf) { return cf; }

__device__ __forceinline__ int div_magic(int a, uint32_t mag, int shf) {
  return (int)(__umulhi((uint32_t)a << 1, mag) >> shf);
}

// descriptor fields of an item with ND dims, in registers
template <int ND>
struct Shape {
  int n[ND], shf[ND];
  uint32_t mag[ND];
  __device__ __forceinline__ explicit Shape(const BoxItem& it) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      n[d] = it.dims[d];
      mag[d] = it.mag[d];
      shf[d] = it.shf[d];
    }
  }
  // multi-index of linear element e (last dim fastest)
  __device__ __forceinline__ void split(int e, int (&t)[ND]) const {
    int rem = e;
#pragma unroll
    for (int d = ND - 1; d > 0; --d) {
      const int q = div_magic(rem, mag[d], shf[d]);
      t[d] = rem - q * n[d];
      rem = q;
    }
    t[0] = rem;
  }
};

template <int ND>
__device__ __forceinline__ int dot(const int (&t)[ND], const int (&s)[ND]) {
  int r = 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) r += t[d] * s[d];
  return r;
}

template <int ND>
__device__ __forceinline__ void load_strides(const int32_t* src, int (&s)[ND]) {
#pragma unroll
  for (int d = 0; d < ND; ++d) s[d] = src[d];
}

// source side of the general form: sum over terms of coef x src[off + ld * a + b]
template <typename TS, typename TD>
struct Src {
  const TS* __restrict__ p;
  const Term* __restrict__ terms;
  int64_t off0, ld0;
  TD c0;
  int nterm, term0;

  __device__ __forceinline__ TD load(int a, int b) const {
    if (nterm == 1) return c0 * TD(__ldg(p + off0 + ld0 * a + b));
    TD acc = TD(0);
    for (int i = 0; i < nterm; ++i) {
      const Term* t = terms + term0 + i;
      acc += coef<TD>(__ldg(&t->coef), __ldg(&t->coef_f)) * TD(__ldg(p + __ldg(&t->off) + __ldg(&t->ld) * a + b));
    }
    return acc;
  }
};

// split-BF16 store: hi = bf16(x) at h[o], lo = bf16(x - hi) at h[o + lo_off]
__device__ __forceinline__ void store_split(__nv_bfloat16* h, int64_t lo_off, int64_t o, float x) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  h[o] = hi;
  h[o + lo_off] = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// destination side of the general form: dst[off + ld * a + b]
template <typename TD>
struct Dst {
  void* p;
  int64_t off, ld, lo_off;
  bool split;
  __device__ __forceinline__ void store(TD v, int a, int b) const {
    const int64_t o = off + ld * a + b;
    if (split)
      store_split(static_cast<__nv_bfloat16*>(p), lo_off, o, (float)v);
    else
      static_cast<TD*>(p)[o] = v;
  }
};

// Lanes past the end of a partial item redo its last element: the same load
// and the same value stored to the same place, so no lane needs a predicate.
template <int ND, typename TS, typename TD>
__device__ __forceinline__ void linear_flat(const BoxItem& it, const TS* __restrict__ src, void* __restrict__ dstv,
                                            int64_t lo_off, int lane) {
  TD* dst = static_cast<TD*>(dstv);
  const Shape<ND> sh(it);
  int sa[ND], da[ND];
  load_strides(it.sa, sa);
  load_strides(it.da, da);
  const TS* ps = src + it.t0_off;
  TD* pd = dst + it.dst_off;
  const int last = it.start + it.count - 1;
  if (it.nterm == 0) {  // zero fill: nothing to read
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      int t[ND];
      sh.split(min(it.start + lane + 32 * u, last), t);
      pd[dot(t, da)] = TD(0);
    }
    return;
  }
  const TD c = coef<TD>(it.t0_coef, it.t0_coef_f);
  TD v[kBatch];
  int dof[kBatch];
#pragma unroll
  for (int u = 0; u < kBatch; ++u) {
    int t[ND];
    sh.split(min(it.start + lane + 32 * u, last), t);
    dof[u] = dot(t, da);
    v[u] = TD(__ldg(ps + dot(t, sa)));
  }
  if (((it.sel >> 4) & 7) == DST_SPLIT) {
    __nv_bfloat16* ph = static_cast<__nv_bfloat16*>(dstv) + it.dst_off;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) store_split(ph, lo_off, dof[u], (float)(c * v[u]));
    return;
  }
#pragma unroll
  for (int u = 0; u < kBatch; ++u) pd[dof[u]] = c * v[u];
}

template <int ND, typename TS, typename TD>
__device__ __forceinline__ void linear_general(const BoxItem& it, const Src<TS, TD>& src, const Dst<TD>& dst,
                                               int lane) {
  const Shape<ND> sh(it);
  const int last = it.start + it.count - 1;
  TD v[kBatch];
  {
    int sa[ND], sb[ND];
    load_strides(it.sa, sa);
    load_strides(it.sb, sb);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      int t[ND];
      sh.split(min(it.start + lane + 32 * u, last), t);
      v[u] = src.load(dot(t, sa), dot(t, sb));
    }
  }
  int da[ND], db[ND];
  load_strides(it.da, da);
  load_strides(it.db, db);
#pragma unroll
  for (int u = 0; u < kBatch; ++u) {
    int t[ND];
    sh.split(min(it.start + lane + 32 * u, last), t);
    dst.store(v[u], dot(t, da), dot(t, db));
  }
}

// one 32 x 32 tile (origin p0, q0) of the last two dims at outer index
// it.start (p: destination-contiguous, q: source-contiguous)
template <typename TS, typename TD>
__device__ __forceinline__ void tile_item(const BoxItem& it, const TS* __restrict__ fsrc, TD* __restrict__ fdst,
                                          const Src<TS, TD>& src, const Dst<TD>& dst, TD (*tile)[33], int lane) {
  const int nd = it.ndim;
  const int P = it.dims[nd - 2], Q = it.dims[nd - 1];
  int rem = it.start, sa = 0, sb = 0, da = 0, db = 0;
#pragma unroll 1
  for (int d = nd - 3; d >= 0; --d) {
    const int q = d > 0 ? div_magic(rem, it.mag[d], it.shf[d]) : 0;
    const int t = rem - q * it.dims[d];
    rem = q;
    sa += t * it.sa[d];
    sb += t * it.sb[d];
    da += t * it.da[d];
    db += t * it.db[d];
  }
  const bool flat = (it.sel & kSelFlat) != 0;
  const int sap = it.sa[nd - 2], saq = it.sa[nd - 1], sbp = it.sb[nd - 2], sbq = it.sb[nd - 1];
  const int dap = it.da[nd - 2], daq = it.da[nd - 1], dbp = it.db[nd - 2], dbq = it.db[nd - 1];
  const int q = it.q0 + lane;
  const int rows = min(32, P - it.p0);
  // two halves of 16 rows: 16 loads per lane in flight, half the registers
#pragma unroll
  for (int h = 0; h < 32; h += 16) {
    TD v[16];
    if (flat) {
      const TS* ps = fsrc + it.t0_off + sa + q * saq + (it.p0 + h) * sap;
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = (h + r < rows && q < Q) ? TD(__ldg(ps + r * sap)) : TD(0);
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int p = it.p0 + h + r;
        v[r] = (h + r < rows && q < Q) ? src.load(sa + p * sap + q * saq, sb + p * sbp + q * sbq) : TD(0);
      }
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) tile[h + r][lane] = v[r];
  }
  __syncwarp();
  const int p = it.p0 + lane;
  const int cols = min(32, Q - it.q0);
  if (p < P) {
    if (flat) {
      const TD c = coef<TD>(it.t0_coef, it.t0_coef_f);
      const int64_t o = it.dst_off + da + (int64_t)p * dap + (int64_t)it.q0 * daq;
      if (dst.split) {
        __nv_bfloat16* ph = static_cast<__nv_bfloat16*>(dst.p);
#pragma unroll 8
        for (int k = 0; k < 32; ++k)
          if (k < cols) store_split(ph, dst.lo_off, o + (int64_t)k * daq, (float)(c * tile[lane][k]));
      } else {
        TD* pd = fdst + o;
#pragma unroll 8
        for (int k = 0; k < 32; ++k)
          if (k < cols) pd[k * daq] = c * tile[lane][k];
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const int qq = it.q0 + k;
        if (k < cols) dst.store(tile[lane][k], da + p * dap + qq * daq, db + p * dbp + qq * dbq);
      }
    }
  }
  __syncwarp();
}

// Fused recoupling item (kSelRecouple): for every position of the box, the
// n_s source values are loaded once and the n_d destinations receive their
// coefficient-weighted sums (Ch. 6, Eq. permsu2, all output labels of one
// set of leg spins at once).  The coefficient matrix is staged in the warp's
// shared-memory tile with rows padded to NS (a bound on n_s: 2, 4, 8 or 16)
// and read back as 8- or 16-byte vectors; the (offset, ld) pairs of sources
// and destinations are staged beside it.  A lane keeps H positions x NS
// values in flight (H * NS about 24 registers of FP32, H at most 8) and the
// destination offsets of its H positions, so items with few sources load
// more positions per round trip; with NS <= 4 the source offsets live in
// registers and every position's loads are issued as soon as its index is
// split.  An item may hold more than 32 positions per lane (the planner
// sizes it by n_s); the lane walks them H at a time.  ND is a bound on the
// box's dims (unused dims are unit).
template <int NS, typename TD>
__device__ __forceinline__ void load_row(const TD* r, TD (&w)[NS]) {
  if constexpr (sizeof(TD) == 4 && NS % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NS; q += 4) {
      const float4 x = *reinterpret_cast<const float4*>(r + q);
      w[q] = x.x;
      w[q + 1] = x.y;
      w[q + 2] = x.z;
      w[q + 3] = x.w;
    }
  } else if constexpr (sizeof(TD) == 4) {
#pragma unroll
    for (int q = 0; q < NS; q += 2) {
      const float2 x = *reinterpret_cast<const float2*>(r + q);
      w[q] = x.x;
      w[q + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NS; q += 2) {
      const double2 x = *reinterpret_cast<const double2*>(r + q);
      w[q] = x.x;
      w[q + 1] = x.y;
    }
  }
}

template <int ND, int NS, typename TS, typename TD>
__device__ __forceinline__ void recouple_item(const BoxItem& it, const Term* __restrict__ terms,
                                              const TS* __restrict__ src, void* dstv, int64_t lo_off, bool split,
                                              TD (*tile)[33], int lane) {
  const int ns = it.nterm, nd = it.p0;
  const Term* T = terms + it.term0;
  TD* cf = &tile[0][0];  // [nd][NS], zero past n_s
  longlong2* sp = reinterpret_cast<longlong2*>(cf + kMaxRecouple * 16);  // (off, ld) of each source
  longlong2* dp = sp + kMaxRecouple;                                       // (off, ld) of each destination
  for (int i = lane; i < nd * NS; i += 32) {
    const int d = i / NS, q = i - d * NS;
    cf[i] = q < ns ? coef<TD>(T[ns + nd + d * ns + q].coef, T[ns + nd + d * ns + q].coef_f) : TD(0);
  }
  if (lane < ns) sp[lane] = make_longlong2(T[lane].off, T[lane].ld);
  if (lane < nd) dp[lane] = make_longlong2(T[ns + lane].off, T[ns + lane].ld);
  __syncwarp();
  const Shape<ND> sh(it);
  int sa[ND], sb[ND];
  load_strides(it.sa, sa);
  load_strides(it.sb, sb);
  const int last = it.start + it.count - 1;
  const int per_lane = (it.count + 31) >> 5;
  int da[ND], db[ND];
  load_strides(it.da, da);
  load_strides(it.db, db);
  // positions in flight per lane: H x NS values and H destination offsets in
  // registers (fewer for 6-dim boxes, whose index split needs more)
  constexpr int kVals = (sizeof(TD) == 4 ? 24 : 16) / (ND > 4 ? 2 : 1);
  constexpr int H = kVals / NS > 8 ? 8 : kVals / NS > 0 ? kVals / NS : 1;
#pragma unroll 1
  for (int u = 0; u < per_lane; u += H) {
    TD v[H][NS];
    int c[H], e[H];  // destination offset parts of each position
    if constexpr (NS <= 4) {
      int64_t so[NS];
      int sl[NS];  // the planner keeps a recoupling item's ld below 2^31
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const longlong2 x = sp[q < ns ? q : 0];
        so[q] = x.x;
        sl[q] = (int)x.y;
      }
#pragma unroll
      for (int h = 0; h < H; ++h) {
        int t[ND];
        sh.split(min(it.start + lane + 32 * (u + h), last), t);
        const int a = dot(t, sa), b = dot(t, sb);
        c[h] = dot(t, da);
        e[h] = dot(t, db);
#pragma unroll
        for (int q = 0; q < NS; ++q)
          v[h][q] = q < ns && u + h < per_lane ? TD(__ldg(src + so[q] + (int64_t)sl[q] * a + b)) : TD(0);
      }
    } else {
      int a[H], b[H];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        int t[ND];
        sh.split(min(it.start + lane + 32 * (u + h), last), t);
        a[h] = dot(t, sa);
        b[h] = dot(t, sb);
        c[h] = dot(t, da);
        e[h] = dot(t, db);
      }
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        if (q < ns) {
          const longlong2 x = sp[q];
          const TS* p = src + x.x;
#pragma unroll
          for (int h = 0; h < H; ++h) v[h][q] = TD(__ldg(p + x.y * a[h] + b[h]));
        } else {
#pragma unroll
          for (int h = 0; h < H; ++h) v[h][q] = TD(0);
        }
      }
    }
#pragma unroll 1
    for (int d = 0; d < nd; ++d) {
      TD w[NS];
      load_row<NS, TD>(cf + d * NS, w);
      const longlong2 x = dp[d];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        if (u + h < per_lane) {  // the item's last positions (warp-uniform)
          TD acc = TD(0);
#pragma unroll
          for (int q = 0; q < NS; ++q) acc = fma(w[q], v[h][q], acc);
          const int64_t o = x.x + x.y * c[h] + e[h];
          if (split)
            store_split(static_cast<__nv_bfloat16*>(dstv), lo_off, o, (float)acc);
          else
            static_cast<TD*>(dstv)[o] = acc;
        }
      }
    }
  }
  __syncwarp();
}

template <typename TS, typename TD>
__device__ __forceinline__ const TS* src_slot(const BoxItem& it, const BoxPtrs& ptrs) {
  const int k = it.sel & 3;
  return static_cast<const TS*>(k == 0 ? ptrs.src[0] : k == 1 ? ptrs.src[1] : k == 2 ? ptrs.src[2] : ptrs.src[3]);
}

__device__ __forceinline__ void* dst_slot(const BoxItem& it, const BoxPtrs& ptrs) {
  switch ((it.sel >> 4) & 7) {
    case 0: return ptrs.dst[0];
    case 1: return ptrs.dst[1];
    case 2: return ptrs.dst[2];
    case 3: return ptrs.dst[3];
    case 4: return ptrs.dst[4];
    default: return ptrs.dst[5];
  }
}

// flat linear item of 4 to 6 dims (rare): the index split reads the descriptor
// from shared memory dim by dim instead of holding it in registers
template <typename TS, typename TD>
__device__ __forceinline__ void linear_flat_rolled(const BoxItem& it, const TS* __restrict__ src,
                                                   void* __restrict__ dstv, int64_t lo_off, int lane) {
  TD* dst = static_cast<TD*>(dstv);
  const TS* ps = src + it.t0_off;
  TD* pd = dst + it.dst_off;
  const int last = it.start + it.count - 1;
  const bool has_src = it.nterm > 0;
  const TD c = coef<TD>(it.t0_coef, it.t0_coef_f);
  TD v[kBatch];
  int dof[kBatch];
#pragma unroll
  for (int u = 0; u < kBatch; ++u) {
    int rem = min(it.start + lane + 32 * u, last), so = 0, dd = 0;
#pragma unroll 1
    for (int d = kMaxDim - 1; d >= 0; --d) {
      const int q = d > 0 ? div_magic(rem, it.mag[d], it.shf[d]) : 0;
      const int t = rem - q * it.dims[d];
      rem = q;
      so += t * it.sa[d];
      dd += t * it.da[d];
    }
    dof[u] = dd;
    v[u] = has_src ? c * TD(__ldg(ps + so)) : TD(0);
  }
  if (((it.sel >> 4) & 7) == DST_SPLIT) {
    __nv_bfloat16* ph = static_cast<__nv_bfloat16*>(dstv) + it.dst_off;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) store_split(ph, lo_off, dof[u], (float)v[u]);
    return;
  }
#pragma unroll
  for (int u = 0; u < kBatch; ++u) pd[dof[u]] = v[u];
}

// flat linear item
template <typename TS, typename TD>
__device__ __forceinline__ void run_flat(const BoxItem& it, const BoxPtrs& ptrs, int lane) {
  const TS* sp = src_slot<TS, TD>(it, ptrs);
  void* d = dst_slot(it, ptrs);
  const int64_t lo = ptrs.split_lo;
  switch (it.ndim) {
    case 1: linear_flat<1, TS, TD>(it, sp, d, lo, lane); break;
    case 2: linear_flat<2, TS, TD>(it, sp, d, lo, lane); break;
    case 3: linear_flat<3, TS, TD>(it, sp, d, lo, lane); break;
    default: linear_flat_rolled<TS, TD>(it, sp, d, lo, lane); break;
  }
}

// recoupling item: dims bound ND and source-count bound NS from the item
template <typename TS, typename TD>
__device__ __forceinline__ void recouple(const BoxItem& it, const Term* __restrict__ terms, const TS* sp, void* dp,
                                         int64_t lo_off, bool split, TD (*tile)[33], int lane) {
  const int ns = it.nterm;
  if (it.ndim <= 4) {
    if (ns <= 2) {
      if (it.ndim <= 2)
        recouple_item<2, 2, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
      else
        recouple_item<4, 2, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
    } else if (ns <= 4) {
      if (it.ndim <= 2)
        recouple_item<2, 4, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
      else
        recouple_item<4, 4, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
    } else if (ns <= 8) {
      recouple_item<4, 8, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
    } else {
      recouple_item<4, 16, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
    }
  } else if (ns <= 8) {
    recouple_item<kMaxDim, 8, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
  } else {
    recouple_item<kMaxDim, 16, TS, TD>(it, terms, sp, dp, lo_off, split, tile, lane);
  }
}

template <typename TS, typename TD>
__device__ __forceinline__ void run_item(const BoxItem& it, const Term* __restrict__ terms, const BoxPtrs& ptrs,
                                         TD (*tile)[33], int lane) {
  if ((it.sel & (kSelFlat | kSelTile)) == kSelFlat) {
    run_flat<TS, TD>(it, ptrs, lane);
    return;
  }
  const TS* sp = src_slot<TS, TD>(it, ptrs);
  void* dp = dst_slot(it, ptrs);
  if (it.sel & kSelRecouple) {
    recouple<TS, TD>(it, terms, sp, dp, ptrs.split_lo, ((it.sel >> 4) & 7) == DST_SPLIT, tile, lane);
    return;
  }
  Src<TS, TD> src;
  src.p = sp;
  src.terms = terms;
  src.off0 = it.t0_off;
  src.ld0 = it.t0_ld;
  src.c0 = coef<TD>(it.t0_coef, it.t0_coef_f);
  src.nterm = it.nterm;
  src.term0 = it.term0;
  Dst<TD> dst;
  dst.p = dp;
  dst.off = it.dst_off;
  dst.ld = it.dst_ld;
  dst.lo_off = ptrs.split_lo;
  dst.split = ((it.sel >> 4) & 7) == DST_SPLIT;
  if (it.sel & kSelTile) {
    tile_item<TS, TD>(it, sp, static_cast<TD*>(dp), src, dst, tile, lane);
    return;
  }
  switch (it.ndim) {
    case 1: linear_general<1, TS, TD>(it, src, dst, lane); break;
    case 2: linear_general<2, TS, TD>(it, src, dst, lane); break;
    case 3: linear_general<3, TS, TD>(it, src, dst, lane); break;
    default: linear_general<kMaxDim, TS, TD>(it, src, dst, lane); break;
  }
}

// Launch variants by the items a launch holds: kBoxGeneral any item;
// kBoxFlat only flat linear items (no tile buffer and a 64-register cap, so
// twice the warps stay resident); kBoxRecouple only flat linear and fused
// recoupling items (no transposing tiles or general sums, so the recoupling
// path is compiled on its own and keeps its loads in registers).
template <typename TS, typename TD, int kMode>
__global__ void __launch_bounds__(kThreads, kMode == kBoxFlat ? 8 : kMode == kBoxRecouple && sizeof(TD) == 4 ? 4 : (sizeof(TD) == 4 ? 5 : 4))
    box_kernel(const BoxItem* __restrict__ items, int nitems, const Term* __restrict__ terms, const BoxPtrs ptrs) {
  __shared__ int64_t raw[kWarps][kItemWords];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nwarps = gridDim.x * kWarps;
  int item = blockIdx.x * kWarps + w;
  if (item >= nitems) return;
  const int64_t* words = reinterpret_cast<const int64_t*>(items);
  int64_t word = lane < kItemWords ? __ldg(words + (int64_t)item * kItemWords + lane) : 0;
  pdl_wait();  // the descriptors are plan constants; the data is not
  pdl_launch_dependents();
  const BoxItem& it = *reinterpret_cast<const BoxItem*>(raw[w]);
  for (; item < nitems; item += nwarps) {
    if (lane < kItemWords) raw[w][lane] = word;
    __syncwarp();
    const int next = item + nwarps;
    if (lane < kItemWords && next < nitems) word = __ldg(words + (int64_t)next * kItemWords + lane);
    if constexpr (kMode == kBoxFlat) {
      run_flat<TS, TD>(it, ptrs, lane);
    } else if constexpr (kMode == kBoxRecouple) {
      __shared__ __align__(16) TD stage[kWarps][32][33];
      if (it.sel & kSelRecouple)
        recouple<TS, TD>(it, terms, src_slot<TS, TD>(it, ptrs), dst_slot(it, ptrs), ptrs.split_lo,
                         ((it.sel >> 4) & 7) == DST_SPLIT, stage[w], lane);
      else
        run_flat<TS, TD>(it, ptrs, lane);
    } else {
      __shared__ __align__(16) TD tiles[kWarps][32][33];
      run_item<TS, TD>(it, terms, ptrs, tiles[w], lane);
    }
    __syncwarp();
  }
}

template <typename TS, typename TD, int kMode>
int launch_t(const BoxItem* items, int nitems, const Term* terms, const BoxPtrs& ptrs, cudaStream_t s) {
  static int slots = 0;  // resident warps of this instantiation on the device
  if (slots == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, box_kernel<TS, TD, kMode>, kThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    slots = per_sm * nsm * kWarps;
  }
  const int warps = nitems < slots ? nitems : slots;
  const int grid = (warps + kWarps - 1) / kWarps;
  return (int)launch_pdl(box_kernel<TS, TD, kMode>, dim3(grid), dim3(kThreads), 0, s, items, nitems, terms, ptrs);
}

template <typename T>
int launch_mode(int mode, const BoxItem* items, int nitems, const Term* terms, const BoxPtrs& ptrs, cudaStream_t s) {
  switch (mode) {
    case kBoxFlat: return launch_t<T, T, kBoxFlat>(items, nitems, terms, ptrs, s);
    case kBoxRecouple: return launch_t<T, T, kBoxRecouple>(items, nitems, terms, ptrs, s);
    default: return launch_t<T, T, kBoxGeneral>(items, nitems, terms, ptrs, s);
  }
}

}  // namespace

int launch_box(bool src_f64, bool dst_f64, int mode, const BoxItem* items, int nitems, const Term* terms,
               const BoxPtrs& ptrs, void* stream) {
  if (nitems <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (src_f64 && dst_f64) return launch_mode<double>(mode, items, nitems, terms, ptrs, s);
  if (!src_f64 && !dst_f64) return launch_mode<float>(mode, items, nitems, terms, ptrs, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace sym
