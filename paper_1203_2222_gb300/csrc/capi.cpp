// C ABI of the library (include/symtensor.h): argument checking, error
// codes, handle ownership.  All work is delegated to structure.cpp (sector
// tables), plan.cpp (work lists) and the CUDA kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <exception>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>

#include "../../include/symtensor.h"
#include "handles.h"
#include "plan.h"
#include "recouple.h"
#include "structure.h"

std::string& sym::last_error() {
  thread_local std::string msg;
  return msg;
}

namespace {

using sym::guard;

void need(bool ok, const char* msg) {
  if (!ok) sym::fail(SYM_ERR_ARG, msg);
}

std::vector<sym::Leg> read_legs(int rank, const sym_leg* legs) {
  need(rank >= 0 && rank <= 6, "rank must be in 0..6");
  need(rank == 0 || legs != nullptr, "legs is NULL");
  std::vector<sym::Leg> out(rank);
  for (int l = 0; l < rank; ++l) {
    need(legs[l].n >= 1 && legs[l].labels && legs[l].degens, "leg needs n >= 1 labels and degeneracies");
    out[l].labels.assign(legs[l].labels, legs[l].labels + legs[l].n);
    out[l].degens.assign(legs[l].degens, legs[l].degens + legs[l].n);
    out[l].dir = legs[l].dir;
  }
  return out;
}

sym::Tree read_tree(int rank, const int* tree) {
  if (!tree) return sym::Tree::comb(rank);
  sym::Tree t;
  t.k = rank;
  for (int n = 0; n + 1 < rank; ++n) t.nodes.push_back({tree[2 * n], tree[2 * n + 1]});
  t.validate();
  return t;
}

void check_precision(int p) {
  need(p == SYM_PREC_FP64 || p == SYM_PREC_BF16X3, "precision must be SYM_PREC_FP64 or SYM_PREC_BF16X3");
}

sym_tensor wrap(sym::Tensor&& t) {
  auto* h = new sym_tensor_s;
  h->t = std::move(t);
  return h;
}

}  // namespace

sym::Tensor sym::contraction_result(const Tensor& a, const Tensor& b, const std::vector<int>& pa,
                                    const std::vector<int>& pb, const int* tree_c) {
  if (a.group != b.group) fail(SYM_ERR_ARG, "A and B belong to different symmetry groups");
  const int npairs = (int)pa.size();
  if (npairs != (int)pb.size() || npairs > std::min(a.rank, b.rank)) fail(SYM_ERR_ARG, "bad number of pairs");
  std::vector<int> sa(a.rank, 0), sb(b.rank, 0);
  for (int i = 0; i < npairs; ++i) {
    if (pa[i] < 0 || pa[i] >= a.rank || sa[pa[i]]) fail(SYM_ERR_ARG, "pairsA: bad or repeated leg");
    if (pb[i] < 0 || pb[i] >= b.rank || sb[pb[i]]) fail(SYM_ERR_ARG, "pairsB: bad or repeated leg");
    sa[pa[i]] = sb[pb[i]] = 1;
    const Leg& la = a.legs[pa[i]];
    const Leg& lb = b.legs[pb[i]];
    if (!la.same_content(lb) || la.dir != -lb.dir)
      fail(SYM_ERR_INCOMPATIBLE_LEGS,
           "contracted legs must carry the same labels and degeneracies with opposite directions");
  }
  std::vector<Leg> legs;
  for (int l = 0; l < a.rank; ++l)
    if (!sa[l]) legs.push_back(a.legs[l]);
  const int na = (int)legs.size();
  for (int l = 0; l < b.rank; ++l)
    if (!sb[l]) legs.push_back(b.legs[l]);
  if (legs.size() > 6) fail(SYM_ERR_ARG, "result rank would exceed 6");
  Tree tr;
  if (sym::su2_like(a.group)) tr = tree_c ? read_tree((int)legs.size(), tree_c) : Tree::comb_pair(na, (int)legs.size() - na);
  return make_tensor(a.group, legs, a.group == SYM_Z2F ? (a.total ^ b.total) : a.total + b.total, tr);
}

namespace {
// FUSE of legs first and first+1 of T: the result structure and the plan
std::pair<sym::Tensor, std::unique_ptr<sym::Plan>> fuse_pair(const sym::Tensor& T, int first, int precision) {
  need(first >= 0 && first + 1 < T.rank, "fuse: first must be in 0..rank-2");
  sym::Leg d = sym::fused_leg(T.legs[first], T.legs[first + 1], T.group);
  std::vector<sym::Leg> legs(T.legs.begin(), T.legs.begin() + first);
  legs.push_back(d);
  legs.insert(legs.end(), T.legs.begin() + first + 2, T.legs.end());
  sym::Tensor O = sym::make_tensor(T.group, legs, T.total, sym::Tree::comb((int)legs.size()));
  auto P = sym::plan_transform(T, O, {}, precision, 1, first);
  return {std::move(O), std::move(P)};
}
}  // namespace

extern "C" {

const char* sym_last_error(void) { return sym::last_error().c_str(); }

const char* sym_version(void) { return "symtensor 0.1 sm_103a"; }

int sym_tensor_create(int group, int rank, const sym_leg* legs, int total, const int* tree, sym_tensor* out) {
  return guard([&] {
    need(out != nullptr, "out is NULL");
    auto L = read_legs(rank, legs);
    sym::Tree tr = sym::su2_like(group) ? read_tree(rank, tree) : sym::Tree{};
    *out = wrap(sym::make_tensor(group, L, total, tr));
    return SYM_OK;
  });
}

int sym_tensor_destroy(sym_tensor t) {
  delete t;
  return SYM_OK;
}

int sym_tensor_info(sym_tensor t, int* group, int* rank, int64_t* numel, int64_t* nsec) {
  return guard([&] {
    need(t != nullptr, "tensor is NULL");
    if (group) *group = t->t.group;
    if (rank) *rank = t->t.rank;
    if (numel) *numel = t->t.numel();
    if (nsec) *nsec = t->t.nsec();
    return SYM_OK;
  });
}

int sym_tensor_leg(sym_tensor t, int leg, int* n, int* labels, int* degens, int* dir) {
  return guard([&] {
    need(t != nullptr && leg >= 0 && leg < t->t.rank, "bad tensor or leg");
    const sym::Leg& L = t->t.legs[leg];
    if (n) *n = (int)L.labels.size();
    if (labels) std::copy(L.labels.begin(), L.labels.end(), labels);
    if (degens) std::copy(L.degens.begin(), L.degens.end(), degens);
    if (dir) *dir = L.dir;
    return SYM_OK;
  });
}

int sym_tensor_tree(sym_tensor t, int* nodes) {
  return guard([&] {
    need(t != nullptr && nodes != nullptr, "NULL argument");
    need(sym::su2_like(t->t.group), "only SU(2) and SU(2) x U(1) tensors have a tree");
    for (size_t n = 0; n < t->t.tree.nodes.size(); ++n) {
      nodes[2 * n] = t->t.tree.nodes[n][0];
      nodes[2 * n + 1] = t->t.tree.nodes[n][1];
    }
    return SYM_OK;
  });
}

int sym_tensor_sectors(sym_tensor t, int* labels, int64_t* offsets) {
  return guard([&] {
    need(t != nullptr, "tensor is NULL");
    const sym::Tensor& T = t->t;
    if (labels) {
      int w = T.rank + T.nin;
      for (int64_t s = 0; s < T.nsec(); ++s) {
        for (int l = 0; l < T.rank; ++l) labels[s * w + l] = T.p(s, l);
        for (int i = 0; i < T.nin; ++i) labels[s * w + T.rank + i] = T.inner_of(s)[i];
      }
    }
    if (offsets) std::copy(T.offs.begin(), T.offs.end(), offsets);
    return SYM_OK;
  });
}

int sym_permute_plan(sym_tensor in, const int* perm, const int* tree_out, int precision, sym_tensor* out,
                     sym_plan* plan) {
  return guard([&] {
    need(in && out && plan, "NULL argument");
    check_precision(precision);
    const sym::Tensor& T = in->t;
    need(T.rank == 0 || perm != nullptr, "perm is NULL");
    std::vector<int> p(perm, perm + T.rank);
    std::vector<int> seen(T.rank, 0);
    for (int x : p) {
      need(x >= 0 && x < T.rank && !seen[x], "perm is not a permutation");
      seen[x] = 1;
    }
    std::vector<sym::Leg> legs;
    for (int x : p) legs.push_back(T.legs[x]);
    sym::Tree tr = sym::su2_like(T.group) ? read_tree(T.rank, tree_out) : sym::Tree{};
    sym::Tensor O = sym::make_tensor(T.group, legs, T.total, tr);
    auto P = sym::plan_transform(T, O, p, precision, 0, 0);
    *out = wrap(std::move(O));
    *plan = new sym_plan_s{std::move(P)};
    return SYM_OK;
  });
}

int sym_fuse_plan(sym_tensor in, int first, int precision, sym_tensor* out, sym_plan* plan) {
  return guard([&] {
    need(in && out && plan, "NULL argument");
    check_precision(precision);
    auto r = fuse_pair(in->t, first, precision);
    *out = wrap(std::move(r.first));
    *plan = new sym_plan_s{std::move(r.second)};
    return SYM_OK;
  });
}

int sym_fuse_n_plan(sym_tensor in, int first, int nlegs, int precision, sym_tensor* out, sym_plan* plan) {
  return guard([&] {
    need(in && out && plan, "NULL argument");
    check_precision(precision);
    const sym::Tensor& T = in->t;
    need(nlegs >= 2 && first >= 0 && first + nlegs <= T.rank, "fuse: legs first..first+nlegs-1 must exist, nlegs >= 2");
    // ((l_first, l_first+1), l_first+2) ...: nlegs - 1 pairwise fuses at `first`
    std::vector<std::unique_ptr<sym::Plan>> steps;
    sym::Tensor cur = T;
    for (int i = 0; i + 1 < nlegs; ++i) {
      auto r = fuse_pair(cur, first, precision);
      cur = std::move(r.first);
      steps.push_back(std::move(r.second));
    }
    std::unique_ptr<sym::Plan> P =
        steps.size() == 1 ? std::move(steps.front()) : sym::chain_transforms(std::move(steps), precision);
    *out = wrap(std::move(cur));
    *plan = new sym_plan_s{std::move(P)};
    return SYM_OK;
  });
}

int sym_split_plan(sym_tensor in, int leg, const sym_leg* parts, int precision, sym_tensor* out, sym_plan* plan) {
  return guard([&] {
    need(in && out && plan && parts, "NULL argument");
    check_precision(precision);
    const sym::Tensor& T = in->t;
    need(leg >= 0 && leg < T.rank, "split: bad leg");
    need(T.rank + 1 <= 6, "split: rank would exceed 6");
    auto ab = read_legs(2, parts);
    sym::Leg d = sym::fused_leg(ab[0], ab[1], T.group);
    const sym::Leg& f = T.legs[leg];
    if (!(d.same_content(f) && d.dir == f.dir))
      sym::fail(SYM_ERR_INCOMPATIBLE_LEGS, "split: the two parts do not fuse to the leg");
    if (sym::su2_like(T.group) && !(T.tree == sym::Tree::comb(T.rank)))
      sym::fail(SYM_ERR_UNSUPPORTED, "split: SU(2) input must be in the comb tree (permute it first)");
    std::vector<sym::Leg> legs(T.legs.begin(), T.legs.begin() + leg);
    legs.push_back(ab[0]);
    legs.push_back(ab[1]);
    legs.insert(legs.end(), T.legs.begin() + leg + 1, T.legs.end());
    sym::Tensor O = sym::make_tensor(T.group, legs, T.total, sym::Tree::comb((int)legs.size()));
    auto P = sym::plan_transform(T, O, {}, precision, 2, leg);
    *out = wrap(std::move(O));
    *plan = new sym_plan_s{std::move(P)};
    return SYM_OK;
  });
}

int sym_plan_execute(sym_plan plan, const void* in, void* out, void* stream) {
  return guard([&] {
    need(plan && plan->p && plan->p->kind == sym::Plan::TRANSFORM, "not a permute/fuse/split plan");
    need((in && out) || plan->p->numel_c == 0, "NULL data pointer");
    return sym::exec_transform(*plan->p, in, out, stream);
  });
}

int sym_contract_plan(sym_tensor A, sym_tensor B, int npairs, const int* pairsA, const int* pairsB,
                      const int* tree_c, int precision, sym_tensor* C, sym_plan* plan) {
  return guard([&] {
    need(A && B && C && plan, "NULL argument");
    check_precision(precision);
    need(npairs >= 0 && (npairs == 0 || (pairsA && pairsB)), "pairs are NULL");
    std::vector<int> pa(pairsA, pairsA + npairs), pb(pairsB, pairsB + npairs);
    sym::Tensor Ct = sym::contraction_result(A->t, B->t, pa, pb, tree_c);
    auto P = sym::plan_contract(A->t, B->t, pa, pb, Ct, precision);
    *C = wrap(std::move(Ct));
    *plan = new sym_plan_s{std::move(P)};
    return SYM_OK;
  });
}

int sym_contract_batch_plan(int nprob, const sym_tensor* A, const sym_tensor* B, int npairs, const int* pairsA,
                            const int* pairsB, int precision, sym_tensor* C, int64_t* offsets, sym_plan* plan) {
  return guard([&] {
    need(nprob >= 1 && A && B && C && offsets && plan, "NULL argument");
    check_precision(precision);
    need(npairs >= 0 && (npairs == 0 || (pairsA && pairsB)), "pairs are NULL");
    for (int i = 0; i < nprob; ++i) need(A[i] && B[i], "NULL tensor in the batch");
    const std::vector<int> pa(pairsA, pairsA + npairs), pb(pairsB, pairsB + npairs);
    std::vector<sym::Tensor> Ct(nprob);
    std::vector<std::unique_ptr<sym::Plan>> ps(nprob);
    // the problems are planned independently, on up to 16 host threads
    std::atomic<int> next{0};
    std::exception_ptr err;
    std::mutex emu;
    auto work = [&] {
      for (int i = next++; i < nprob; i = next++) {
        try {
          Ct[i] = sym::contraction_result(A[i]->t, B[i]->t, pa, pb, nullptr);
          ps[i] = sym::plan_contract(A[i]->t, B[i]->t, pa, pb, Ct[i], precision, /*device=*/false);
        } catch (...) {
          std::lock_guard<std::mutex> lk(emu);
          if (!err) err = std::current_exception();
        }
      }
    };
    const int nth = std::max(1, std::min({nprob, 16, (int)std::thread::hardware_concurrency()}));
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    if (err) std::rethrow_exception(err);
    std::vector<int64_t> oa(nprob + 1, 0), ob(nprob + 1, 0), oc(nprob + 1, 0);
    for (int i = 0; i < nprob; ++i) {
      oa[i + 1] = oa[i] + A[i]->t.numel();
      ob[i + 1] = ob[i] + B[i]->t.numel();
      oc[i + 1] = oc[i] + Ct[i].numel();
    }
    auto M = sym::merge_contract_plans(ps, oa, ob, oc);
    for (int i = 0; i <= nprob; ++i) {
      offsets[i] = oa[i];
      offsets[nprob + 1 + i] = ob[i];
      offsets[2 * (nprob + 1) + i] = oc[i];
    }
    for (int i = 0; i < nprob; ++i) C[i] = wrap(std::move(Ct[i]));
    *plan = new sym_plan_s{std::move(M)};
    return SYM_OK;
  });
}

int sym_contract(sym_plan plan, const void* A, const void* B, void* C, void* stream) {
  return guard([&] {
    need(plan && plan->p && plan->p->kind == sym::Plan::CONTRACT, "not a contraction plan");
    return sym::exec_contract(*plan->p, A, B, C, stream);
  });
}

int sym_contract_backward(sym_plan plan, const void* A, const void* B, const void* dC, void* dA, void* dB,
                          void* stream) {
  return guard([&] {
    need(plan && plan->p && plan->p->kind == sym::Plan::CONTRACT, "not a contraction plan");
    return sym::exec_contract_backward(*plan->p, A, B, dC, dA, dB, stream);
  });
}

int sym_plan_stats(sym_plan plan, double* flops_fwd, int64_t* bytes_a, int64_t* bytes_b, int64_t* bytes_c) {
  return guard([&] {
    need(plan && plan->p, "plan is NULL");
    const sym::Plan& p = *plan->p;
    int64_t es = p.f64() ? 8 : 4;
    if (flops_fwd) *flops_fwd = p.flops_fwd;
    if (bytes_a) *bytes_a = p.numel_a * es;
    if (bytes_b) *bytes_b = p.numel_b * es;
    if (bytes_c) *bytes_c = p.numel_c * es;
    return SYM_OK;
  });
}

int sym_plan_launches(sym_plan plan, int* launches) {
  return guard([&] {
    need(plan && plan->p && launches, "NULL argument");
    *launches = plan->p->last_launches;
    return SYM_OK;
  });
}

int sym_plan_profile(sym_plan plan, int enable) {
  return guard([&] {
    need(plan && plan->p, "plan is NULL");
    if (enable) plan->p->clear_profile();
    plan->p->profiling = enable != 0;
    return SYM_OK;
  });
}

namespace {
// device time of one recorded launch (waits for its end event)
double launch_ms(const sym::LaunchRecord& e) {
  cudaError_t err = cudaEventSynchronize(static_cast<cudaEvent_t>(e.e1));
  if (err != cudaSuccess) sym::fail(SYM_ERR_CUDA, std::string("event: ") + cudaGetErrorString(err));
  float t = 0.f;
  cudaEventElapsedTime(&t, static_cast<cudaEvent_t>(e.e0), static_cast<cudaEvent_t>(e.e1));
  return t;
}
}  // namespace

int sym_plan_profile_read(sym_plan plan, int phase, int* launches, double* total_ms, double* bytes, double* flops) {
  return guard([&] {
    need(plan && plan->p, "plan is NULL");
    need(phase >= 0 && phase < sym::PH_COUNT, "bad phase");
    sym::PhaseProfile& pp = plan->p->prof[phase];
    double ms = 0.0;
    for (auto& e : pp.events) ms += launch_ms(e);
    if (launches) *launches = pp.launches;
    if (total_ms) *total_ms = ms;
    if (bytes) *bytes = pp.bytes;
    if (flops) *flops = pp.flops;
    return SYM_OK;
  });
}

int sym_plan_profile_kernel(sym_plan plan, int kernel, int* launches, double* total_ms, double* bytes,
                            double* flops) {
  return guard([&] {
    need(plan && plan->p, "plan is NULL");
    need(kernel >= 0 && kernel < SYM_KERNEL_COUNT, "bad kernel");
    int n = 0;
    double ms = 0.0, by = 0.0, fl = 0.0;
    for (const sym::PhaseProfile& pp : plan->p->prof)
      for (const auto& e : pp.events)
        if (e.kernel == kernel) {
          ++n;
          ms += launch_ms(e);
          by += e.bytes;
          fl += e.flops;
        }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    if (bytes) *bytes = by;
    if (flops) *flops = fl;
    return SYM_OK;
  });
}

int sym_tune_get(sym_tune* out) {
  return guard([&] {
    need(out != nullptr, "NULL argument");
    *out = sym::current_tune();
    return SYM_OK;
  });
}

int sym_tune_set(const sym_tune* in) {
  return guard([&] {
    need(in != nullptr, "NULL argument");
    sym::set_tune(*in);
    return SYM_OK;
  });
}

int sym_tune_epoch(int* epoch) {
  return guard([&] {
    need(epoch != nullptr, "NULL argument");
    *epoch = sym::tune_epoch();
    return SYM_OK;
  });
}

int sym_plan_gemm_shapes(sym_plan plan, int* nsec, int* mnk) {
  return guard([&] {
    need(plan && plan->p && nsec, "NULL argument");
    const sym::Plan& p = *plan->p;
    // one entry per GEMM sector: tensor-core sectors, then CUDA-core sectors
    std::vector<std::array<int, 4>> v;
    for (const auto& s : p.secs_tc) v.push_back({s.m, s.n, s.k, 0});
    for (const auto& s : p.secs_simt) v.push_back({s.m, s.n, s.k, 1});
    if (mnk)
      for (size_t i = 0; i < v.size(); ++i)
        for (int j = 0; j < 4; ++j) mnk[4 * i + j] = v[i][j];
    *nsec = (int)v.size();
    return SYM_OK;
  });
}

int sym_plan_destroy(sym_plan plan) {
  delete plan;
  return SYM_OK;
}

int sym_su2_F(int jd, int je, int ja, int jb, int jc, int J, double* out) {
  return guard([&] {
    need(out != nullptr, "out is NULL");
    for (int v : {jd, je, ja, jb, jc, J}) need(v >= 0 && v <= 60, "spins must be in 0..60 (doubled)");
    *out = sym::recoupF(jd, je, ja, jb, jc, J);
    return SYM_OK;
  });
}

int sym_su2_gamma(int rank, const int* spins, const int* tree_in, const int* perm, const int* tree_out, int* n_in,
                  int* n_out, double* G, int* labels_in, int* labels_out) {
  return guard([&] {
    need(rank >= 0 && rank <= 6 && (rank == 0 || (spins && perm)), "bad rank, spins or perm");
    std::vector<int> sp(spins, spins + rank), p(perm, perm + rank), seen(rank, 0);
    for (int x : p) {
      need(x >= 0 && x < rank && !seen[x], "perm is not a permutation");
      seen[x] = 1;
    }
    for (int s : sp) need(s >= 0 && s <= 60, "spins must be in 0..60 (doubled)");
    sym::Tree ti = read_tree(rank, tree_in), to = read_tree(rank, tree_out);
    sym::Gamma g = sym::tree_transform(sp, ti, p, to);
    if (n_in) *n_in = (int)g.in_labels.size();
    if (n_out) *n_out = (int)g.out_labels.size();
    if (G) std::copy(g.G.begin(), g.G.end(), G);
    const int w = std::max(rank - 2, 0);
    if (labels_in)
      for (size_t i = 0; i < g.in_labels.size(); ++i) std::copy(g.in_labels[i].begin(), g.in_labels[i].end(), labels_in + i * w);
    if (labels_out)
      for (size_t o = 0; o < g.out_labels.size(); ++o)
        std::copy(g.out_labels[o].begin(), g.out_labels[o].end(), labels_out + o * w);
    return SYM_OK;
  });
}

int sym_device_status(void) {
  return guard([&] {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) sym::fail(SYM_ERR_CUDA, std::string("device: ") + cudaGetErrorString(e));
    int code = sym::take_device_error();
    if (code != SYM_OK)
      sym::fail(code, code == SYM_ERR_NUMERIC ? "an SVD block did not converge" : "a bounded device-side wait expired");
    return SYM_OK;
  });
}

int sym_wait_probe(int limit_us, int word) {
  return guard([&] {
    if (limit_us < 1 || limit_us > 2000000 || (word != 0 && word != 1))
      sym::fail(SYM_ERR_ARG, "sym_wait_probe: limit_us in 1..2000000, word 0 or 1");
    int* w = word == 0 ? sym::device_error_word() : sym::noalloc_error_word();
    int e = sym::launch_wait_probe(w, (uint64_t)limit_us * 1000ull, nullptr);
    if (e == 0) e = (int)cudaDeviceSynchronize();
    if (e != 0) sym::fail(SYM_ERR_CUDA, std::string("wait probe: ") + cudaGetErrorString((cudaError_t)e));
    return SYM_OK;
  });
}

}  // extern "C"
