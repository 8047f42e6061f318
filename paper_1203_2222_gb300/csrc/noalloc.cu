// Contraction for callers that cannot allocate device memory.
//
// sym_contract / sym_contract_plan keep their work lists and operand scratch
// in device buffers obtained with cudaMalloc when the plan is created.  Some
// callers cannot do that -- code that runs where the CUDA allocator must not
// be entered (inside a host callback, under an allocation-free real-time
// budget, next to a framework that owns every byte of device memory) -- so
// this entry point runs the same contraction out of one file-scope device
// array instead.  Its plans are built on the host only and cached under the
// contents of the two structures (never their handle addresses, which the
// allocator reuses once a handle is destroyed); every call copies the work
// lists into the array with cudaMemcpyAsync and launches the same gather /
// GEMM / scatter kernels as sym_contract.  Nothing in the array needs to
// start at zero: the gathers write every operand element the GEMMs read,
// the plan's zero-fill items clear the outputs that split reductions add
// into, and the tensor cores' loads get their zeros past the operand edges
// from the tensor maps' out-of-bounds fill, as in the regular path.
#include <cuda_runtime.h>

#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "handles.h"

namespace sym {
namespace {

constexpr size_t kNoallocBytes = size_t(32) << 20;  // 32 MiB of device scratch

// Static device scratch shared by every call on a device; it keeps the last
// call's contents.  Host code must not use its name as a device address:
// the address comes from cudaGetSymbolAddress (scratch_base below).
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];
// Error word of the bounded device-side waits of this entry point's
// launches; sym_device_status reads and clears it with the library's own.
__device__ int g_noalloc_err;

constexpr size_t kMaxPlans = 64;  // cached plans; the oldest is dropped beyond this

std::mutex g_mu;
struct DeviceSyms {
  unsigned char* scratch;
  int* err;
};
std::map<int, DeviceSyms> g_syms;  // device -> addresses of the two arrays

// Contents of a structure that its plans depend on: group, total label,
// legs (labels, degeneracies, direction) and fusion tree.
void fingerprint(const Tensor& t, std::vector<int>& k) {
  k.push_back(t.group);
  k.push_back(t.rank);
  k.push_back(t.total);
  for (const Leg& l : t.legs) {
    k.push_back((int)l.labels.size());
    k.push_back(l.dir);
    k.insert(k.end(), l.labels.begin(), l.labels.end());
    k.insert(k.end(), l.degens.begin(), l.degens.end());
  }
  k.push_back((int)t.tree.nodes.size());
  for (const auto& n : t.tree.nodes) {
    k.push_back(n[0]);
    k.push_back(n[1]);
  }
}

// cache key: both structures, the pairs, the precision and the planning
// parameters' epoch (a plan built under older parameters is not reused)
std::vector<int> plan_key(const Tensor& a, const Tensor& b, const std::vector<int>& pa, const std::vector<int>& pb,
                          int precision) {
  std::vector<int> k;
  fingerprint(a, k);
  fingerprint(b, k);
  k.push_back((int)pa.size());
  k.insert(k.end(), pa.begin(), pa.end());
  k.insert(k.end(), pb.begin(), pb.end());
  k.push_back(precision);
  k.push_back(tune_epoch());
  return k;
}
std::map<std::vector<int>, std::unique_ptr<Plan>> g_plans;
std::deque<std::vector<int>> g_order;  // insertion order of g_plans' keys

// Device addresses of the static arrays on the current device, looked up
// once per device with that device current.
DeviceSyms device_syms() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  auto it = g_syms.find(dev);
  if (it != g_syms.end()) return it->second;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    fail(SYM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
  void* q = nullptr;
  e = cudaGetSymbolAddress(&q, g_noalloc_err);
  if (e != cudaSuccess || q == nullptr)
    fail(SYM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static error word: ") + cudaGetErrorString(e));
  DeviceSyms d{static_cast<unsigned char*>(p), static_cast<int*>(q)};
  register_device_error_word(d.err);
  g_syms[dev] = d;
  return d;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int* noalloc_error_word() { return device_syms().err; }

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
    std::vector<int> key = plan_key(A->t, B->t, pa, pb, precision);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
      Tensor Ct = contraction_result(A->t, B->t, pa, pb, nullptr);
      auto plan = plan_contract(A->t, B->t, pa, pb, Ct, precision, /*device=*/false);
      plan->concurrent = false;  // no side streams or events: launch the GEMM kinds in order
      if (g_plans.size() >= kMaxPlans) {
        g_plans.erase(g_order.front());
        g_order.pop_front();
      }
      it = g_plans.emplace(key, std::move(plan)).first;
      g_order.push_back(key);
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
    const size_t o_img = region((size_t)p.img_elems * 2 * 2);  // hi and lo planes
    const size_t o_lin = region((size_t)p.lin_elems * es);
    const size_t o_outm = region((size_t)p.outm_elems * es);
    if (off > kNoallocBytes)
      fail(SYM_ERR_UNSUPPORTED, "sym_contract_noalloc: this contraction needs " + std::to_string(off) +
                                    " bytes of scratch, above the static limit of " + std::to_string(kNoallocBytes) +
                                    " bytes (use sym_contract)");
    const DeviceSyms syms = device_syms();
    unsigned char* base = syms.scratch;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto copy = [&](size_t o, const void* h, size_t bytes) {
      if (!bytes) return;
      cudaError_t e = cudaMemcpyAsync(base + o, h, bytes, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
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
    // The array keeps the previous call's contents, and nothing here relies
    // on zeros in it (see the head of this file).  The error word is left
    // as it is: sym_device_status reads and clears it.
    p.d_items = reinterpret_cast<BoxItem*>(base + o_items);
    p.d_terms = reinterpret_cast<Term*>(base + o_terms);
    p.d_ditems = reinterpret_cast<DirectItem*>(base + o_ditems);
    p.d_secs_simt = reinterpret_cast<GemmSectorSimt*>(base + o_simt);
    p.d_secs_tc = reinterpret_cast<TcSector*>(base + o_tc);
    p.d_tiles = reinterpret_cast<GemmTile*>(base + o_tiles);
    p.d_maps = reinterpret_cast<TensorMap*>(base + o_maps);
    p.d_err = syms.err;
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
