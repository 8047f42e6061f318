// Execution plans: the precomputed, structure-only part of every operation.
#pragma once

#include <memory>
#include <vector>

#include "kernels.h"
#include "structure.h"
#include "../../include/symtensor.h"

namespace sym {

struct Range {
  int first = 0, count = 0;
};

// Owner of the device allocations of one plan.
struct DeviceArena {
  std::vector<void*> ptrs;
  void* alloc(size_t bytes, bool zero);
  ~DeviceArena();
};

// Phases of a plan's launches (profiling and statistics).
enum Phase { PH_FWD_GATHER = 0, PH_FWD_GEMM, PH_FWD_SCATTER, PH_BWD_GATHER, PH_BWD_GEMM, PH_BWD_SCATTER,
             PH_XFORM, PH_FWD_GEMM_SIMT, PH_BWD_GEMM_SIMT, PH_FWD_DIRECT, PH_BWD_DIRECT, PH_COUNT };
constexpr int kGemmKinds = 5;  // 0 tcgen05, CUDA cores: 1 tile 64x64, 2 tile 256x16, 3 thin, 4 rows

// One recorded launch: cudaEvent_t pair around it, kernel (SYM_KERNEL_*),
// algorithmic bytes and useful flops.
struct LaunchRecord {
  void* e0;
  void* e1;
  int kernel;
  double bytes, flops;
};
struct PhaseProfile {
  std::vector<LaunchRecord> events;
  int launches = 0;
  double bytes = 0.0, flops = 0.0;  // algorithmic, summed over the recorded launches
};

struct Plan {
  enum Kind { TRANSFORM = 1, CONTRACT = 2 };
  int kind = 0;
  int precision = 0;  // SYM_PREC_*
  bool f64() const;

  // box work lists of every phase, in one uploaded array
  std::vector<BoxItem> items;
  std::vector<Term> terms;
  Range xform;                        // TRANSFORM: in -> out
  // TRANSFORM made of several transforms run in order (a fuse of more than
  // two legs: pairwise fuses), through two plan-owned scratch buffers
  std::vector<std::unique_ptr<Plan>> chain;
  void* chain_buf[2] = {nullptr, nullptr};
  Range fwd_gather, fwd_scatter;      // CONTRACT forward
  Range bwd_gather_a, bwd_gather_b;   // backward gathers needed for dA / dB
  Range bwd_scatter_a, bwd_scatter_b;

  // direct-contraction work lists (sectors with a tiny matrix on one side,
  // see kernels.h), their columns inline
  std::vector<DirectItem> ditems;
  Range fwd_direct, bwd_direct_a, bwd_direct_b;  // C = A B; dA = dC B^T; dB += A^T dC
  std::vector<double> ditem_bytes_prefix, ditem_flops_prefix;  // launch statistics

  // GEMM work lists.  Kinds: 0 = tcgen05 split-BF16 x3, 1 = CUDA-core 64x64,
  // 2 = CUDA-core 256x16, 3 = CUDA-core thin (m, n <= 8), 4 = CUDA-core
  // rows (k, n <= 16); GEMM phases:
  // 0 = forward, 1 = dA, 2 = dB.
  std::vector<GemmSectorSimt> secs_simt;
  std::vector<TcSector> secs_tc;
  std::vector<GemmTile> tiles;  // grouped by kind, then by GEMM phase
  Range gemm_range[kGemmKinds][3];  // [kind][gemm phase]
  std::vector<int> tile_kind;   // kind of every tile (statistics)
  std::vector<TcOperand> tc_ops;  // split-BF16 operands of the tcgen05 GEMMs
  std::vector<TensorMap> maps;    // their tensor maps (encoded for the image buffer at maps_base)
  const void* maps_base = nullptr;
  void encode_maps(const void* img_base);

  // scratch sizes (elements): split-BF16 images, linear operands, output matrices
  int64_t img_elems = 0, lin_elems = 0, outm_elems = 0;

  // statistics
  double flops_fwd = 0.0;
  int64_t numel_a = 0, numel_b = 0, numel_c = 0;
  int last_launches = 0;
  bool dry = false;  // built with SYM_PLAN_DRYRUN=1: validated on the host, never uploaded

  // algorithmic bytes of every box item and useful flops of every tile,
  // as prefix sums (launch statistics for any range in O(1))
  std::vector<double> item_bytes_prefix, tile_flops_prefix, tile_bytes_prefix;
  std::vector<int> flat_prefix;      // flat linear items among the first i (launch variant choice)
  std::vector<int> recouple_prefix;  // fused recoupling items among the first i
  void set_item_bytes(Range r, int es_src, int es_dst);
  bool profiling = false;
  PhaseProfile prof[PH_COUNT];
  void clear_profile();
  ~Plan();

  // device copies
  DeviceArena arena;
  BoxItem* d_items = nullptr;
  Term* d_terms = nullptr;
  DirectItem* d_ditems = nullptr;
  GemmSectorSimt* d_secs_simt = nullptr;
  TcSector* d_secs_tc = nullptr;
  GemmTile* d_tiles = nullptr;
  TensorMap* d_maps = nullptr;
  void* img = nullptr;     // split-BF16 operands: hi plane, then lo plane img_elems further
  void* lin = nullptr;     // linear operands (fp32 or fp64)
  void* outm = nullptr;    // output matrices (fp32 or fp64)
  int* d_err = nullptr;

  // The GEMM kinds of one phase touch disjoint sectors: they are forked onto
  // side streams and joined back (created on first use; events and streams
  // are captured into a CUDA graph as dependencies).  Off for plans that
  // must create nothing (sym_contract_noalloc).
  bool concurrent = true;
  int tc_order = 0;  // tcgen05 tiles: 0 longest reduction first, 1 in sector order
  // The backward reads the tensor-core operands the forward gathered when
  // bwd_reads_fwd_operands; they are reused if the plan's last forward ran
  // on the same A and B buffers, and gathered again otherwise.
  bool bwd_reads_fwd_operands = false;
  const void* fwd_a = nullptr;
  const void* fwd_b = nullptr;
  void* side[kGemmKinds - 1] = {};     // cudaStream_t
  void* ev_fork = nullptr;             // cudaEvent_t
  void* ev_join[kGemmKinds - 1] = {};  // cudaEvent_t

  void validate(const int64_t* src_elems, const int64_t* dst_elems) const;
  void upload(bool device = true);
};

// planning parameters (sym_tune of the C ABI): read at plan time
sym_tune current_tune();
void set_tune(const sym_tune& t);  // validated; bumps the epoch
int tune_epoch();

std::unique_ptr<Plan> plan_transform(const Tensor& in, const Tensor& out, const std::vector<int>& perm,
                                     int precision, int mode_fuse_split, int leg);
// a transform made of the given ones run in order (each one's output the
// next one's input); owns two scratch buffers for the intermediates
std::unique_ptr<Plan> chain_transforms(std::vector<std::unique_ptr<Plan>> steps, int precision);
// device = false builds and validates the work lists on the host only (no
// device allocation); such a plan runs only through sym_contract_noalloc.
std::unique_ptr<Plan> plan_contract(const Tensor& A, const Tensor& B, const std::vector<int>& pairsA,
                                    const std::vector<int>& pairsB, const Tensor& C, int precision,
                                    bool device = true);
// many independent contractions as one plan over packed buffers (see plan.cpp)
std::unique_ptr<Plan> merge_contract_plans(std::vector<std::unique_ptr<Plan>>& ps, const std::vector<int64_t>& offA,
                                           const std::vector<int64_t>& offB, const std::vector<int64_t>& offC,
                                           bool device = true);

// Execution (asynchronous on `stream`); return SYM_OK or a negative code.
int exec_transform(Plan& p, const void* in, void* out, void* stream);
int exec_contract(Plan& p, const void* A, const void* B, void* C, void* stream);
int exec_contract_backward(Plan& p, const void* A, const void* B, const void* dC, void* dA, void* dB,
                           void* stream);

// Device error word written by bounded waits (SYM_OK or SYM_ERR_TIMEOUT);
// take_device_error() reads and clears it.
int* device_error_word();
int take_device_error();
// Another device error word (a static __device__ int) that take_device_error
// also reads and clears.
void register_device_error_word(int* w);
// sym_contract_noalloc's static error word on the current device (noalloc.cu).
int* noalloc_error_word();

// Structure helpers shared with the C ABI.
Leg fused_leg(const Leg& a, const Leg& b, int group);
Tree fuse_pair_tree(int k, int f);  // node (f, f+1) first, then the comb over the k-1 items

}  // namespace sym
