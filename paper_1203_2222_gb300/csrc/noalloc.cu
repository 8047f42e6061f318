// Contraction for callers that cannot allocate device memory.
//
// sym_contract / sym_contract_plan keep their work lists and operand scratch
// in device buffers obtained with cudaMalloc when the plan is created.  Some
// callers cannot do that -- code that runs where the CUDA allocator must not
// be entered (inside a host callback, under an allocation-free real-time
// budget, next to a framework that owns every byte of device memory) -- so
// this entry point runs the same contraction out of one file-scope device
// array instead.  Its plans are built on the host only and cached; every
// call copies the work lists into the array with cudaMemcpyAsync, clears the
// regions that must start at zero with cudaMemsetAsync, and launches the
// same gather / GEMM / scatter kernels as sym_contract.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "handles.h"

namespace sym {
namespace {

constexpr size_t kNoallocBytes = size_t(32) << 20;  // 32 MiB of device scratch

// Static device scratch shared by every call on a device; it keeps the last
// call's contents.  Host code must not use its name as a device address:
// the address comes from cudaGetSymbolAddress (scratch_base below).
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
std::map<int, unsigned char*> g_base;  // device -> address of g_noalloc_scratch
using PlanKey = std::tuple<const void*, const void*, std::vector<int>, std::vector<int>, int>;
std::map<PlanKey, std::unique_ptr<Plan>> g_plans;

// Device address of the static array on the current device (set up once per
// device, with that device current).
unsigned char* scratch_base() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  auto it = g_base.find(dev);
  if (it != g_base.end()) return it->second;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    fail(SYM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
  g_base[dev] = static_cast<unsigned char*>(p);
  return g_base[dev];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace sym

extern "C" int sym_contract_noalloc(sym_tensor A, sym_tensor B, int npairs, const int* pairsA, const int* pairsB,
                                    int precision, const void* a, const void* b, void* c, void* stream) {
  using namespace sym;
  return guard([&] {
    if (!A || !B) fail(SYM_ERR_ARG, "NULL tensor");
    if (precision != SYM_PREC_FP64 && precision != SYM_PREC_BF16X3)
      fail(SYM_ERR_ARG, "precision must be SYM_PREC_FP64 or SYM_PREC_BF16X3");
    if (npairs < 0 || (npairs > 0 && (!pairsA || !pairsB))) fail(SYM_ERR_ARG, "bad pairs");
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<int> pa(pairsA, pairsA + npairs), pb(pairsB, pairsB + npairs);
    PlanKey key{A, B, pa, pb, precision};
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
      Tensor Ct = contraction_result(A->t, B->t, pa, pb, nullptr);
      it = g_plans.emplace(key, plan_contract(A->t, B->t, pa, pb, Ct, precision, /*device=*/false)).first;
      it->second->concurrent = false;  // no side streams or events: launch the GEMM kinds in order
    }
    Plan& p = *it->second;
    if (!a || !b || (p.numel_c > 0 && !c)) fail(SYM_ERR_ARG, "NULL data pointer");
    // layout of the static array for this plan
    const size_t es = p.f64() ? sizeof(double) : sizeof(float);
    size_t off = 0;
    auto region = [&](size_t bytes) {
      const size_t o = off;
      off = align256(off + bytes);
      return o;
    };
    const size_t o_items = region(p.items.size() * sizeof(BoxItem));
    const size_t o_terms = region(p.terms.size() * sizeof(Term));
    const size_t o_ditems = region(p.ditems.size() * sizeof(DirectItem));
    const size_t o_simt = region(p.secs_simt.size() * sizeof(GemmSectorSimt));
    const size_t o_tc = region(p.secs_tc.size() * sizeof(TcSector));
    const size_t o_tiles = region(p.tiles.size() * sizeof(GemmTile));
    const size_t o_maps = region(p.tc_ops.size() * sizeof(TensorMap));
    const size_t o_err = region(sizeof(int));
    const size_t o_img = region((size_t)p.img_elems * 2 * 2);  // hi and lo planes
    const size_t o_lin = region((size_t)p.lin_elems * es);
    const size_t o_outm = region((size_t)p.outm_elems * es);
    if (off > kNoallocBytes)
      fail(SYM_ERR_UNSUPPORTED, "sym_contract_noalloc: this contraction needs " + std::to_string(off) +
                                    " bytes of scratch, above the static limit of " + std::to_string(kNoallocBytes) +
                                    " bytes (use sym_contract)");
    unsigned char* base = scratch_base();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto copy = [&](size_t o, const void* h, size_t bytes) {
      if (!bytes) return;
      cudaError_t e = cudaMemcpyAsync(base + o, h, bytes, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    };
    auto zero = [&](size_t o, size_t bytes) {
      if (!bytes) return;
      cudaError_t e = cudaMemsetAsync(base + o, 0, bytes, s);
      if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    };
    copy(o_items, p.items.data(), p.items.size() * sizeof(BoxItem));
    copy(o_terms, p.terms.data(), p.terms.size() * sizeof(Term));
    copy(o_ditems, p.ditems.data(), p.ditems.size() * sizeof(DirectItem));
    copy(o_simt, p.secs_simt.data(), p.secs_simt.size() * sizeof(GemmSectorSimt));
    copy(o_tc, p.secs_tc.data(), p.secs_tc.size() * sizeof(TcSector));
    copy(o_tiles, p.tiles.data(), p.tiles.size() * sizeof(GemmTile));
    if (!p.tc_ops.empty()) {  // tensor maps point into this array: encode them for its address
      p.encode_maps(base + o_img);
      copy(o_maps, p.maps.data(), p.maps.size() * sizeof(TensorMap));
    }
    // the array keeps the previous call's contents: clear what must start at
    // zero (the TMA loads of the tensor cores read zeros past the operand edges)
    zero(o_err, sizeof(int));
    p.d_items = reinterpret_cast<BoxItem*>(base + o_items);
    p.d_terms = reinterpret_cast<Term*>(base + o_terms);
    p.d_ditems = reinterpret_cast<DirectItem*>(base + o_ditems);
    p.d_secs_simt = reinterpret_cast<GemmSectorSimt*>(base + o_simt);
    p.d_secs_tc = reinterpret_cast<TcSector*>(base + o_tc);
    p.d_tiles = reinterpret_cast<GemmTile*>(base + o_tiles);
    p.d_maps = reinterpret_cast<TensorMap*>(base + o_maps);
    p.d_err = reinterpret_cast<int*>(base + o_err);
    p.img = base + o_img;
    p.lin = base + o_lin;
    p.outm = base + o_outm;
    p.dry = false;
    int rc;
    try {
      rc = exec_contract(p, a, b, c, stream);
    } catch (...) {
      p.dry = true;
      throw;
    }
    p.dry = true;
    return rc;
  });
}
