// Grouped per-sector GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Blockwise matrix multiply of Ch. 5, Eq. blockmult: C_x = A_x B_x for every
// sector x of a contraction (and of many contractions) in one persistent
// launch.  FP32-accurate split-BF16: every FP32 operand is stored as
// hi = bf16(a), lo = bf16(a - hi) and the product is accumulated in FP32 in
// tensor memory as  A_hi B_hi + A_hi B_lo + A_lo B_hi  (3 passes).
//
// Operands arrive as row-major bf16 matrices (hi and lo planes) written by the
// gather (box.cu); the TMA engine loads 128-row x 64-k boxes of them through
// 3-D tensor maps (k, row, plane) with 128-byte swizzling, which is the
// canonical K-major layout of the tensor-core shared-memory descriptors, and
// fills boxes past the matrix edges with zeros.
//
// Roles (192 threads, one CTA per SM, persistent over the tile list):
//   warp 0     one thread issues the TMA tensor loads into a 3-stage ring;
//   warp 1     allocates 256 TMEM columns (two 128x128 FP32 accumulators),
//              one thread issues tcgen05.mma (M=128, N=128, K=16);
//   warps 2-5  epilogue: tcgen05.ld of the accumulator, transpose through
//              shared memory, coalesced FP32 stores; frees the accumulator.
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on expiry the
// CTA sets the device error word and leaves its loops, waits (bounded) for
// its outstanding copies and MMAs, and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/symtensor.h"
#include "kernels.h"
#include "pdl.h"

namespace sym {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int STAGES = 3;
constexpr int TILE_BYTES = 128 * 64 * 2;  // one 128-row x 64-k bf16 box
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A_hi, A_lo, B_hi, B_lo
constexpr int EPI_PITCH = 33;
constexpr int EPI_BYTES = 4 * 32 * EPI_PITCH * 4;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_BYTES + BAR_BYTES;
constexpr int NUM_THREADS = 192;
constexpr uint32_t TMEM_COLS = 256;
// instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A bf16 (7-9 = 1),
// B bf16 (10-12 = 1), both K-major, N>>3 at bits 17-22, M>>4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint64_t WAIT_NS = 2000000000ull;
// The tensor pipe accumulates at most KCHUNK k-tiles (512 of the reduction)
// in one TMEM accumulator; the epilogue adds the chunks in FP32 registers with
// round-to-nearest.  Long in-pipe accumulations measured an error growing
// with k (1.5e-5 relative at k = 4096); per-chunk folding keeps it flat.
constexpr int KCHUNK = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// one box of a 3-D tensor map at (x, y, z) into shared memory
__device__ __forceinline__ void tma_load_3d(void* sdst, const TensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(sdst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1 (bits 46-47), layout type
// SWIZZLE_128B = 2 (bits 61-63).  LBO is unused for swizzled K-major.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// MN-major, 128-byte swizzle: rows of 64 MN elements (128 bytes) along K,
// 8-row K groups 1024 bytes apart (SBO), the two 64-wide MN halves of the
// 128-wide tile 8192 bytes apart (LBO).  Every address an MMA of K = 16
// touches stays inside the 16 KB tile.
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(8192 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// one operand tile (128 rows of the M or N dim x 64 of K) of k-tile kt: a
// K-major map yields it in one 64 x 128 box, an MN-major map in two 64 x 64
// boxes (the MN halves, 8 KB apart)
__device__ __forceinline__ void load_operand(uint8_t* sp, const TensorMap* map, bool mn, int row0, int kt, int plane,
                                             uint64_t* bar);

__device__ __forceinline__ void load_operand(uint8_t* sp, const TensorMap* map, bool mn, int row0, int kt, int plane,
                                             uint64_t* bar) {
  if (mn) {  // x = MN offset (128-byte aligned), y = k
    tma_load_3d(sp, map, row0, kt * 64, plane, bar);
    tma_load_3d(sp + TILE_BYTES / 2, map, row0 + 64, kt * 64, plane, bar);
  } else {   // x = k offset (128-byte aligned), y = row
    tma_load_3d(sp, map, kt * 64, row0, plane, bar);
  }
}

struct Ctl {
  volatile int abort;
};

// Bounded wait; false on timeout or when another role aborted.
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, Ctl* ctl, int* err, uint64_t limit_ns = WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (ctl->abort) return false;
    if (now_ns() - t0 > limit_ns) {
      ctl->abort = 1;
      atomicExch(err, SYM_ERR_TIMEOUT);
      return false;
    }
  }
}

// Bounded wait used on the way out: never sets abort, gives up silently.
__device__ void drain_bar(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (now_ns() - t0 > WAIT_NS) return;
  }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    gemm_tc_kernel(const TcSector* __restrict__ secs, const GemmTile* __restrict__ tiles, int ntiles,
                   const TensorMap* __restrict__ maps, float* __restrict__ C, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* stages = smem;
  float* epi = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + EPI_BYTES);
  uint64_t* full = bars;                // [STAGES]
  uint64_t* empty = bars + STAGES;      // [STAGES]
  uint64_t* tfull = bars + 2 * STAGES;  // [2]
  uint64_t* tempty = tfull + 2;         // [2]
  uint64_t* mma_done = tempty + 2;      // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  Ctl* ctl = reinterpret_cast<Ctl*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);
    }
    mbar_init(mma_done, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_wait();  // barriers and tensor memory are set up; operands and C belong to earlier kernels
  pdl_launch_dependents();

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        const GemmTile t = tiles[ti];
        const TcSector s = secs[t.sector];
        for (int kt = 0; kt < s.ktiles; ++kt) {
          if (!wait_bar(&empty[stage], phase ^ 1u, ctl, err)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
          uint8_t* sp = stages + stage * STAGE_BYTES;
          load_operand(sp, maps + s.amap, s.a_mn, t.mt * BM, kt, 0, &full[stage]);
          load_operand(sp + TILE_BYTES, maps + s.amap, s.a_mn, t.mt * BM, kt, 1, &full[stage]);
          load_operand(sp + 2 * TILE_BYTES, maps + s.bmap, s.b_mn, t.nt * BN, kt, 0, &full[stage]);
          load_operand(sp + 3 * TILE_BYTES, maps + s.bmap, s.b_mn, t.nt * BN, kt, 1, &full[stage]);
          ++issued;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA can exit
        for (int i = 1; i <= STAGES && i <= issued; ++i) {
          int s = stage - i;
          uint32_t ph = phase;
          if (s < 0) {
            s += STAGES;
            ph ^= 1u;
          }
          drain_bar(&full[s], ph);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        const GemmTile t = tiles[ti];
        const TcSector s = secs[t.sector];
        // one TMEM accumulator per chunk of KCHUNK k-tiles, alternating buffers
        for (int k0 = 0; k0 < s.ktiles && ok; k0 += KCHUNK) {
          if (!wait_bar(&tempty[acc], aphase ^ 1u, ctl, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
          const int k1 = min(s.ktiles, k0 + KCHUNK);
          // transpose bits: A MN-major (bit 15), B MN-major (bit 16)
          const uint32_t idesc = IDESC | ((uint32_t)(s.a_mn != 0) << 15) | ((uint32_t)(s.b_mn != 0) << 16);
          for (int kt = k0; kt < k1; ++kt) {
            if (!wait_bar(&full[stage], phase, ctl, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(stages + stage * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // k advances 16: 32 bytes along a K-major row, two 8-row groups MN-major
              const uint64_t ah = s.a_mn ? sw128_mn_desc(base + kk * 2048) : sw128_desc(base + kk * 32);
              const uint64_t al = s.a_mn ? sw128_mn_desc(base + TILE_BYTES + kk * 2048)
                                         : sw128_desc(base + TILE_BYTES + kk * 32);
              const uint64_t bh = s.b_mn ? sw128_mn_desc(base + 2 * TILE_BYTES + kk * 2048)
                                         : sw128_desc(base + 2 * TILE_BYTES + kk * 32);
              const uint64_t bl = s.b_mn ? sw128_mn_desc(base + 3 * TILE_BYTES + kk * 2048)
                                         : sw128_desc(base + 3 * TILE_BYTES + kk * 32);
              mma_bf16(d_tmem, ah, bh, idesc, (kt != k0 || kk != 0) ? 1u : 0u);
              mma_bf16(d_tmem, ah, bl, idesc, 1u);
              mma_bf16(d_tmem, al, bh, idesc, 1u);
            }
            mma_commit(&empty[stage]);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          mma_commit(&tfull[acc]);
          acc ^= 1;
          if (acc == 0) aphase ^= 1u;
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(mma_done);
      drain_bar(mma_done, 0);
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    float* buf = epi + (warp - 2) * 32 * EPI_PITCH;
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      const GemmTile t = tiles[ti];
      const TcSector s = secs[t.sector];
      // a small sector fills part of the tile: rows past m and 32-column
      // chunks past n are neither read from TMEM nor stored
      const int row_base = t.mt * BM + q * 32;
      const bool rows_live = row_base < s.m;
      const int ncols = min(BN, s.n - t.nt * BN);
      // this thread's row of the 128 x 128 tile, summed over the k chunks
      float racc[BN];
#pragma unroll
      for (int i = 0; i < BN; ++i) racc[i] = 0.0f;
      for (int k0 = 0; k0 < s.ktiles; k0 += KCHUNK) {
        if (!wait_bar(&tfull[acc], aphase, ctl, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (rows_live) {
#pragma unroll
          for (int c = 0; c < BN; c += 32) {
            if (c >= ncols) break;
            uint32_t r[32];
            tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c), r);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i) racc[c + i] += __uint_as_float(r[i]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        acc ^= 1;
        if (acc == 0) aphase ^= 1u;
      }
      if (!ok) break;
      if (!rows_live) continue;
      // transpose through shared memory: coalesced row segments of C
      const int nrows = min(32, s.m - row_base);
#pragma unroll
      for (int c = 0; c < BN; c += 32) {
        if (c >= ncols) break;
        const int col0 = t.nt * BN + c;
#pragma unroll
        for (int i = 0; i < 32; ++i) buf[lane * EPI_PITCH + i] = racc[c + i];
        __syncwarp();
        const int col = col0 + lane;
        if (col < s.n)
          for (int rr = 0; rr < nrows; ++rr)
            C[s.c_off + (int64_t)(row_base + rr) * s.ldc + col] = s.alpha * buf[rr * EPI_PITCH + lane];
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

int g_num_sms = 0;

// One bounded wait, on the path the kernel's waits take, for the phase of
// an mbarrier that nothing arrives at: it expires after limit_ns and sets
// SYM_ERR_TIMEOUT in *err.  Lets a test check the expiry path and the error
// word without a fault or a hang.
__global__ void wait_probe_kernel(int* err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ Ctl ctl;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    ctl.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) wait_bar(&bar, 0u, &ctl, err, limit_ns);
}

}  // namespace

int launch_wait_probe(int* err_word, uint64_t limit_ns, void* stream) {
  if (limit_ns > WAIT_NS) limit_ns = WAIT_NS;
  wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(err_word, limit_ns);
  return (int)cudaGetLastError();
}

int tc_num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

int launch_gemm_tc(const TcSector* secs, const GemmTile* tiles, int ntiles, const TensorMap* maps, float* C,
                   int* err_word, void* stream) {
  if (ntiles <= 0) return 0;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  int grid = ntiles < tc_num_sms() ? ntiles : tc_num_sms();
  return (int)launch_pdl(gemm_tc_kernel, dim3(grid), dim3(NUM_THREADS), SMEM_BYTES, static_cast<cudaStream_t>(stream),
                         secs, tiles, ntiles, maps, C, err_word);
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}
}  // namespace

int encode_operand_map(TensorMap* out, const void* hi, const TcOperand& op, int64_t split_lo) {
  static_assert(sizeof(TensorMap) == sizeof(CUtensorMap), "TensorMap must hold a CUtensorMap");
  EncodeTiled fn = encode_fn();
  if (!fn) return (int)CUDA_ERROR_NOT_FOUND;
  const cuuint64_t dims[3] = {(cuuint64_t)op.cols, (cuuint64_t)op.rows, 2};
  const cuuint64_t strides[2] = {(cuuint64_t)op.ld * 2, (cuuint64_t)split_lo * 2};  // bytes, dims 1 and 2
  // K-major: 64 k x 128 rows; MN-major: 64 of the M/N dim x 64 k (two per tile)
  const cuuint32_t box[3] = {64, op.mn ? 64u : (cuuint32_t)BM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  void* base = const_cast<uint16_t*>(static_cast<const uint16_t*>(hi) + op.off);
  return (int)fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}


}  // namespace sym
