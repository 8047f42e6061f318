// Execution plans: the precomputed, structure-only part of every operation.
#pragma once

#include <memory>
#include <vector>

#include "kernels.h"
#include "structure.h"

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

struct Plan {
  enum Kind { TRANSFORM = 1, CONTRACT = 2 };
  int kind = 0;
  int precision = 0;  // SYM_PREC_*
  bool f64() const;

  // box work lists of every phase, in one uploaded array
  std::vector<BoxItem> items;
  std::vector<Term> terms;
  Range xform;                        // TRANSFORM: in -> out
  Range fwd_gather, fwd_scatter;      // CONTRACT forward
  Range bwd_gather_a, bwd_gather_b;   // backward gathers needed for dA / dB
  Range bwd_scatter_a, bwd_scatter_b;

  // GEMM work lists (one of the two sector kinds is used)
  std::vector<GemmSector64> secs64;
  std::vector<TcSector> secs_tc;
  std::vector<GemmTile> tiles;
  Range fwd_tiles, bwd_tiles_a, bwd_tiles_b;

  // scratch sizes (elements): operands (bf16 pairs or fp64) and output matrices
  int64_t ops_elems = 0, outm_elems = 0;

  // statistics
  double flops_fwd = 0.0;
  int64_t numel_a = 0, numel_b = 0, numel_c = 0;
  int last_launches = 0;
  bool dry = false;  // built with SYM_PLAN_DRYRUN=1: validated on the host, never uploaded

  // device copies
  DeviceArena arena;
  BoxItem* d_items = nullptr;
  Term* d_terms = nullptr;
  void* d_secs = nullptr;
  GemmTile* d_tiles = nullptr;
  void* ops0 = nullptr;  // fp64 operands, or bf16 hi images
  void* ops1 = nullptr;  // bf16 lo images
  void* outm = nullptr;  // fp32 / fp64 output matrices
  int* d_err = nullptr;

  void validate(const int64_t* src_elems, const int64_t* dst_elems, bool dst0_image) const;
  void upload();
};

std::unique_ptr<Plan> plan_transform(const Tensor& in, const Tensor& out, const std::vector<int>& perm,
                                     int precision, int mode_fuse_split, int leg);
std::unique_ptr<Plan> plan_contract(const Tensor& A, const Tensor& B, const std::vector<int>& pairsA,
                                    const std::vector<int>& pairsB, const Tensor& C, int precision);

// Execution (asynchronous on `stream`); return SYM_OK or a negative code.
int exec_transform(Plan& p, const void* in, void* out, void* stream);
int exec_contract(Plan& p, const void* A, const void* B, void* C, void* stream);
int exec_contract_backward(Plan& p, const void* A, const void* B, const void* dC, void* dA, void* dB,
                           void* stream);

// Device error word written by bounded waits (SYM_OK or SYM_ERR_TIMEOUT);
// take_device_error() reads and clears it.
int* device_error_word();
int take_device_error();

// Structure helpers shared with the C ABI.
Leg fused_leg(const Leg& a, const Leg& b, int group);
Tree fuse_pair_tree(int k, int f);  // node (f, f+1) first, then the comb over the k-1 items

}  // namespace sym
