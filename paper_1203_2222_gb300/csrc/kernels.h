// Device work descriptors shared by the host planner and the CUDA kernels.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define SYM_HD __host__ __device__
#else
#define SYM_HD
#endif

namespace sym {

constexpr int kMaxDim = 6;

// Destination slots of a box launch.
// DST_SPLIT: split-BF16 operands of the tensor cores; an element v goes to
// dst[DST_SPLIT] as hi = bf16(v) and, split_lo elements further, as
// lo = bf16(v - hi) (both rounded to nearest).
enum DstSlot { DST_OUT = 0, DST_DA = 1, DST_DB = 2, DST_OPS = 3, DST_OUTM = 4, DST_SPLIT = 5, DST_COUNT = 6 };
constexpr int kSelTile = 1 << 9;   // BoxItem::sel flag: 32 x 32 transposing tile (see box.cu)
// BoxItem::sel flag: at most one term with t0_ld == 1, linear destination with
// dst_ld == 1, sb == db == 0, and both <t, sa> and <t, da> below 2^31, so the
// kernel addresses source and destination with one 32-bit dot product each
constexpr int kSelFlat = 1 << 10;
constexpr int kSelUnit = 1 << 11;  // BoxItem::sel flag: one term whose coefficient is exactly 1
// BoxItem::sel flag: fused recoupling item.  nterm = n_s sources and p0 = n_d
// destinations share the box; terms[term0 .. term0 + n_s) are the sources
// (src[off + ld <t, sa> + <t, sb>]), the next n_d the destinations
// (dst[off + ld <t, da> + <t, db>]), then the n_d x n_s coefficients
// (row-major, in coef / coef_f): destination d receives
// sum_s coef[d][s] source_s.  Each source element is read once for all d.
constexpr int kSelRecouple = 1 << 12;
constexpr int kMaxRecouple = 16;  // largest n_s and n_d of a fused recoupling item
constexpr int kBoxChunk = 512;  // elements of a linear work item (32 lanes x 16)

// One work unit of the block-movement kernel: a strided box of `dims`
// (last dim fastest) whose element t is
//   dst  <- sum over terms  coef * src[term.off + term.ld * <t, sa> + <t, sb>]
// written to dst[dst_off + dst_ld * <t, da> + <t, db>].
// Only elements [start, start + count) of the box (row-major linear index)
// belong to this unit; the planner guarantees that every destination element
// is written by exactly one unit.  An item with no terms writes zeros.
// Tile items (kSelTile) instead cover outer indices [start, start + count)
// of dims[0..ndim-2) times one 32 x 32 tile (origin p0, q0) of the last two
// dims, whose last is the source's contiguous one and whose second-to-last is
// the destination's.
struct BoxItem {
  int64_t t0_off, t0_ld;  // first term, inline (no second round trip when nterm == 1)
  double t0_coef;
  int64_t dst_off;
  int32_t dst_ld;   // multiplier of <t, da>
  int32_t sel;      // source slot (bits 0-1), destination slot (bits 4-6), kSel* flags
  int32_t ndim;
  int32_t term0, nterm;
  int32_t start, count;
  int32_t p0, q0;  // tile items: origin of the 32 x 32 tile in the last two dims
  int32_t dims[kMaxDim];
  int32_t sa[kMaxDim], sb[kMaxDim];
  int32_t da[kMaxDim], db[kMaxDim];
  // Dims d >= ndim hold size 1 with zero strides, so a kernel may treat the
  // box as having more dims than it does.
  // division by dims[d] without a divide: for 0 <= a < 2^31,
  // floor(a / dims[d]) = umulhi(2a, mag[d]) >> shf[d] (Granlund & Montgomery,
  // PLDI 1994, Thm 4.2 with N = 31: shf = ceil(log2 dims), mag = ceil(2^(31+shf) / dims))
  uint32_t mag[kMaxDim];
  int8_t shf[kMaxDim];
  int8_t pad_[2];
  float t0_coef_f;  // t0_coef rounded to FP32 (the FP32 kernels issue no FP64 instruction)
};
static_assert(sizeof(BoxItem) == 224, "BoxItem layout");

struct Term {
  int64_t off;
  int64_t ld;
  double coef;
  float coef_f;  // coef rounded to FP32 (set by the planner)
  int32_t pad_;
};

// Buffers a box launch may read (src slots) and write (dst slots).
struct BoxPtrs {
  const void* src[4];
  void* dst[DST_COUNT];
  int64_t split_lo;  // DST_SPLIT: element distance from the hi to the lo plane
};

// CUDA-core grouped GEMM (row-major): C = alpha * A (m x k, lda) * B (k x n, ldb).
// trans bit 0: A is stored transposed, element (i, kk) at a[kk * lda + i];
// bit 1: B is stored transposed, element (kk, j) at b[j * ldb + kk] (the
// backward reads the forward's operands this way instead of gathering
// transposed copies).  The rows kernel takes bit 1 only and needs lda == k,
// ldc == n; the thin kernel takes both; the tile kernels neither.
struct GemmSectorSimt {
  int32_t m, n, k, lda, ldb, ldc;
  int64_t a_off, b_off, c_off;
  double alpha;
  int32_t trans, pad_;
};
constexpr int kTransA = 1, kTransB = 2;
// One output tile; [k0, k1) is its slice of the reduction (split-K tiles of
// one sector add into a zero-filled C with atomics when `atomic` is set).
// Rows kernel: [k0, k1) are the tile's rows of C instead (the reduction is
// always whole there), and a tile is the work of one warp.
struct GemmTile {
  int32_t sector, mt, nt;
  int32_t k0, k1, atomic;
};
// Rows kernel: a warp stages kRowsSpan consecutive elements of A (whole rows,
// rows_span(k) of them) in shared memory per step; a tile is kRowsSpansPerTile steps.
constexpr int kRowsSpan = 512;
constexpr int kRowsSpansPerTile = 8;
SYM_HD inline int rows_span(int k) { return (kRowsSpan / k) & ~31; }  // k <= 16: >= 32 rows

// tcgen05 split-BF16 x3 grouped GEMM, C (m x n, row-major FP32, ldc) =
// alpha A B.  The operands are row-major bf16 matrices with their hi and lo
// planes split_lo elements apart, each described by a TensorMap (amap, bmap
// index the plan's map array: 3-D tiled maps (inner, outer, plane) whose
// boxes the TMA engine writes to shared memory in the 128-byte-swizzled
// layouts of the tensor-core descriptors, with zeros past the edges).
// a_mn = 0: A stored m x k (K-major, 64 x 128 boxes of (k, row));
// a_mn = 1: A stored k x m (MN-major, 64 x 64 boxes of (m, k), two per tile).
// b_mn = 0: B stored as B^T, n x k (K-major); b_mn = 1: B stored k x n.
struct TcSector {
  int32_t m, n, k, ktiles;
  int32_t amap, bmap;
  int32_t a_mn, b_mn;
  int64_t c_off;
  int32_t ldc;
  float alpha;
};
struct alignas(64) TensorMap {  // opaque CUtensorMap (128 bytes)
  uint64_t w[16];
};
// Operand of a tensor-core GEMM: a rows x cols bf16 matrix at element `off`
// of the hi plane (row stride ld and off multiples of 64).  mn = 0: K-major
// (rows = the M or N dim, cols = K); mn = 1: MN-major (rows = K, cols = the
// M or N dim).  One buffer may carry one map of each kind.
struct TcOperand {
  int64_t off;
  int32_t rows, cols, ld, mn;
};

// Direct contraction of a sector whose matrix on one side is tiny (k, n <=
// kMaxDirect): the GEMM runs on the tensors' blocks themselves, with no
// matrix form.  An item is a chunk [start, start + count) of the positions t
// of a row group's box (the free legs of the large operand, ndim <= 3 dims,
// last fastest).  Its columns are inline: source column s holds, at
// position t, the element at src_slot + src[s].off + <t, src[s].str>, and
// destination column d the element at dst + dst[d].off + <t, dst[d].str>.
//   apply: dst_d[t] = sum_s kc[d][s] * slot2[koff[d][s]] * src_s[t]       (C = A B, dA = dC B^T)
//   outer: out(s, d) = sum_t src_s[t] * slot2_d[t], the d columns read from
//          slot 2; kc[d][s] * out(s, d) is added (atomically) to the
//          destination slot at koff[d][s]                                (dB = A^T dC)
// kc == 0 marks a structurally absent coefficient.  An item is 512 bytes,
// one 16-byte load per lane.
constexpr int kMaxDirect = 4;
constexpr int kDirectDims = 3;
constexpr int kDirectApplyChunk = 1024;  // default positions per apply item
enum DirectOp { kDirectApply = 0, kDirectOuter = 1 };
struct DirectCol {
  int64_t off;
  int32_t str[kDirectDims];
  int32_t pad_;
};
struct DirectItem {
  int32_t op, ns, nd, ndim;
  int32_t start, count;
  int32_t slots;  // bits 0-1 source slot, 2-3 second source slot, 4-6 destination slot
  int32_t shf;    // the three division shifts, one byte each
  int32_t dims[kDirectDims];
  uint32_t mag[kDirectDims];  // Granlund-Montgomery division by dims[d] (as in BoxItem)
  int32_t pad_[2];
  DirectCol src[kMaxDirect], dst[kMaxDirect];
  int64_t koff[kMaxDirect * kMaxDirect];  // [d * kMaxDirect + s]
  double kc[kMaxDirect * kMaxDirect];
};
static_assert(sizeof(DirectCol) == 24, "DirectCol layout");
static_assert(sizeof(DirectItem) == 512, "DirectItem layout");

// CUDA-core GEMM tile shapes
enum SimtShape { SIMT_64x64 = 0, SIMT_256x16 = 1, SIMT_THIN = 2, SIMT_ROWS = 3, SIMT_SHAPES = 4 };

// Launchers (return cudaError_t as int).
// mode: the items the launch holds, which picks the kernel variant.
// kBoxGeneral: any item; kBoxFlat: only flat linear items (kSelFlat without
// kSelTile); kBoxRecouple: only flat linear and fused recoupling items.
constexpr int kBoxGeneral = 0, kBoxFlat = 1, kBoxRecouple = 2;
int launch_box(bool src_f64, bool dst_f64, int mode, const BoxItem* items, int nitems, const Term* terms,
               const BoxPtrs& ptrs, void* stream);
int launch_gemm_simt(bool f64, int shape, const GemmSectorSimt* secs, const GemmTile* tiles, int ntiles,
                     const void* ops, void* outm, void* stream);
// every item of [items, items + nitems) must have op == `op`
int launch_direct(bool f64, int op, const DirectItem* items, int nitems, const BoxPtrs& ptrs, void* stream);
int launch_gemm_tc(const TcSector* secs, const GemmTile* tiles, int ntiles, const TensorMap* maps, float* C,
                   int* err_word, void* stream);
// One bounded mbarrier wait that nothing completes (a test of the expiry
// path): sets SYM_ERR_TIMEOUT in *err_word after limit_ns (at most the
// kernels' own 2 s limit).
int launch_wait_probe(int* err_word, uint64_t limit_ns, void* stream);
// Tensor map of one operand whose hi plane starts at `hi` (bf16) and whose lo
// plane is split_lo elements further; 0 or a CUDA driver error code.
int encode_operand_map(TensorMap* out, const void* hi, const TcOperand& op, int64_t split_lo);
int tc_num_sms();

}  // namespace sym
