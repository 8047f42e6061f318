// Device work descriptors shared by the host planner and the CUDA kernels.
#pragma once

#include <cstdint>

namespace sym {

constexpr int kMaxDim = 6;

// Destination slots of a box launch.
enum DstSlot { DST_OUT = 0, DST_DA = 1, DST_DB = 2, DST_OPS = 3, DST_OUTM = 4, DST_COUNT = 5 };
constexpr int kSelTile = 1 << 9;   // BoxItem::sel flag: 32 x 32 transposing tile (see box.cu)
// BoxItem::sel flag: at most one term with t0_ld == 1, linear destination with
// dst_ld == 1, sb == db == 0, and both <t, sa> and <t, da> below 2^31, so the
// kernel addresses source and destination with one 32-bit dot product each
constexpr int kSelFlat = 1 << 10;
constexpr int kSelUnit = 1 << 11;  // BoxItem::sel flag: one term whose coefficient is exactly 1
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
};

// CUDA-core grouped GEMM (row-major): C = alpha * A (m x k, lda) * B (k x n, ldb).
struct GemmSectorSimt {
  int32_t m, n, k, lda, ldb, ldc;
  int64_t a_off, b_off, c_off;
  double alpha;
};
// One output tile; [k0, k1) is its slice of the reduction (split-K tiles of
// one sector add into a zero-filled C with atomics when `atomic` is set).
struct GemmTile {
  int32_t sector, mt, nt;
  int32_t k0, k1, atomic;
};

// tcgen05 split-BF16 x3 grouped GEMM.  Operand images: A tile (mt, kt) at
// a_img + (mt * ktiles + kt) * 8192 bf16 elements (128 rows x 64 k, 128B
// swizzled), B tile (nt, kt) likewise with n rows.  C row-major fp32.
// The images are made from FP32 row-major matrices by the pack kernel, one
// PackTile per image tile: rows [128 mt, 128 mt + 128) and columns
// [64 kt, 64 kt + 64) of the rows x cols matrix at src (row stride ld),
// zero outside it, written as the hi and lo images of tile (mt, kt) of the
// operand image at img (ktiles tiles per row tile).
struct TcSector {
  int32_t m, n, k, ktiles;
  int64_t a_img, b_img;
  int64_t c_off;
  int32_t ldc;
  float alpha;
};
struct PackTile {
  int64_t src, img;
  int32_t rows, cols, ld, ktiles, mt, kt;
};

// CUDA-core GEMM tile shapes
enum SimtShape { SIMT_64x64 = 0, SIMT_256x16 = 1, SIMT_THIN = 2, SIMT_ROWS = 3, SIMT_SHAPES = 4 };

// Launchers (return cudaError_t as int).
// flat_only: every item is a flat linear item (kSelFlat without kSelTile)
int launch_box(bool src_f64, bool dst_f64, bool flat_only, const BoxItem* items, int nitems, const Term* terms,
               const BoxPtrs& ptrs, void* stream);
int launch_gemm_simt(bool f64, int shape, const GemmSectorSimt* secs, const GemmTile* tiles, int ntiles,
                     const void* ops, void* outm, void* stream);
int launch_gemm_tc(const TcSector* secs, const GemmTile* tiles, int ntiles, const uint16_t* a_hi,
                   const uint16_t* a_lo, const uint16_t* b_hi, const uint16_t* b_lo, float* C,
                   int* err_word, void* stream);
int launch_pack(const PackTile* tiles, int ntiles, const float* lin, uint16_t* hi, uint16_t* lo, void* stream);
int tc_num_sms();

}  // namespace sym
