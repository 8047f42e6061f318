// Planner: turns tensor structures into device work lists (host, integer
// exact apart from the FP64 recoupling coefficients).
//
// A contraction (Ch. 5 "Multiplication of two tensors", steps 1-5; Ch. 6 for
// tree decompositions) is planned as
//   A --(permute free legs first; SU(2): Gamma to the matrix tree)--> A_mat
//   B --(permute contracted legs first; SU(2): Gamma)---------------> B_mat
//   per sector x:  C_x = A_x B_x   (blockwise product, Ch. 5 Eq. blockmult)
//   C_x --(split rows/cols into blocks; SU(2): Gamma to the output tree)--> C
// A_mat (B_mat) is a tensor whose legs are [rows..., cols...] and whose SU(2)
// tree is a comb over the row legs and a comb over the column legs joined at
// the root, so a sector x is the spin on the two subtrees (U(1): the fused
// charge of the contracted legs).  Inside sector x, row groups (one per
// labelling of the row subtree) and column groups are stacked in
// lexicographic order of their labels; the same rule on both operands makes
// A's columns and B's rows coincide.
//
// SU(2) normalisation.  With cups on incoming legs (Ch. 6) and the root
// vertex C_{x,x->0} = omega_x (Ch. 5, Eq. singletomega), contracting the
// column subtree of A with the row subtree of B leaves, per sector,
//   C_x = (-1)^(2x) / sqrt(2x+1) * prod_{paired legs incoming in A} (-1)^(2j)
//         * A_x B_x
// (the cup on a paired leg passes through a splitting vertex unchanged when
// both sides share the subtree; a cup on A's side is the transpose,
// cup_j^T = (-1)^(2j) cup_j).  The factor is folded into A's gather.
#include "plan.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <cstdlib>
#include <mutex>
#include <set>
#include <string>

#include "../../include/symtensor.h"
#include "recouple.h"

namespace sym {

namespace {

constexpr int kChunk = kBoxChunk;  // elements of a linear box work item
using TermList = std::vector<std::pair<int64_t, double>>;

struct Box {
  int ndim = 0;
  int dims[kMaxDim], sa[kMaxDim], sb[kMaxDim], da[kMaxDim], db[kMaxDim];
  void push(int d, int a, int b, int c, int e) {
    dims[ndim] = d;
    sa[ndim] = a;
    sb[ndim] = b;
    da[ndim] = c;
    db[ndim] = e;
    ++ndim;
  }
};

// drop unit dims and merge dims that are contiguous in all four mappings
Box simplify(const Box& in) {
  Box b;
  for (int i = 0; i < in.ndim; ++i) {
    if (in.dims[i] == 1) continue;
    if (b.ndim > 0) {
      int j = b.ndim - 1;
      int d = in.dims[i];
      if ((int64_t)b.sa[j] == (int64_t)in.sa[i] * d && (int64_t)b.sb[j] == (int64_t)in.sb[i] * d &&
          (int64_t)b.da[j] == (int64_t)in.da[i] * d && (int64_t)b.db[j] == (int64_t)in.db[i] * d) {
        b.dims[j] *= d;
        b.sa[j] = in.sa[i];
        b.sb[j] = in.sb[i];
        b.da[j] = in.da[i];
        b.db[j] = in.db[i];
        continue;
      }
    }
    b.push(in.dims[i], in.sa[i], in.sb[i], in.da[i], in.db[i]);
  }
  if (b.ndim == 0) b.push(1, 0, 0, 0, 0);
  return b;
}

// Magic numbers for dividing 31-bit dividends by d >= 1 with one multiply-high
// (Granlund & Montgomery, PLDI 1994, Thm 4.2 with N = 31):
// s = ceil(log2 d), m = ceil(2^(31+s) / d) < 2^32, floor(a / d) = (2a * m) >> (32 + s).
void div_magic(int d, uint32_t& m, int8_t& s) {
  int l = 0;
  while (((int64_t)1 << l) < d) ++l;
  m = (uint32_t)((((uint64_t)1 << (31 + l)) + (uint64_t)d - 1) / (uint64_t)d);
  s = (int8_t)l;
}

BoxItem make_item(const Box& box, int64_t dst_off, int dst_ld, int sel, int term0,
                  const std::vector<Term>& terms) {
  BoxItem it{};
  it.dst_off = dst_off;
  it.dst_ld = dst_ld;
  it.sel = sel;
  it.ndim = box.ndim;
  it.term0 = term0;
  it.nterm = (int)terms.size();
  if (!terms.empty()) {
    it.t0_off = terms[0].off;
    it.t0_ld = terms[0].ld;
    it.t0_coef = terms[0].coef;
    it.t0_coef_f = (float)terms[0].coef;
  }
  for (int i = 0; i < box.ndim; ++i) {
    it.dims[i] = box.dims[i];
    it.sa[i] = box.sa[i];
    it.sb[i] = box.sb[i];
    it.da[i] = box.da[i];
    it.db[i] = box.db[i];
    div_magic(box.dims[i], it.mag[i], it.shf[i]);
  }
  for (int i = box.ndim; i < kMaxDim; ++i) {
    it.dims[i] = 1;
    div_magic(1, it.mag[i], it.shf[i]);
  }
  if (terms.size() == 1 && terms[0].coef == 1.0) it.sel |= kSelUnit;
  return it;
}

// Emit the work items of one box.  When the source's contiguous dimension is
// not the destination's, the box is cut into 32 x 32 transposing tiles over
// (destination-contiguous dim, source-contiguous dim); otherwise into linear
// chunks of kChunk elements.
void emit(Plan& P, const Box& box0, int64_t dst_off, int dst_ld, int src_slot, int dst_slot,
          const std::vector<Term>& terms0) {
  int sel = src_slot | (dst_slot << 4);
  // Flat form: with at most one term and a linear destination, fold the
  // two-part offsets (ld * a + b) into one stride per dim on each side when
  // every offset of the box stays below 2^31.
  Box box = box0;
  std::vector<Term> terms = terms0;
  if (terms.size() <= 1) {
    const int64_t ld0 = terms.empty() ? 0 : terms[0].ld;
    Box f;
    int64_t sspan = 0, dspan = 0;
    bool ok = true;
    for (int d = 0; d < box0.ndim; ++d) {
      const int64_t s = terms.empty() ? 0 : ld0 * box0.sa[d] + box0.sb[d];
      const int64_t t = (int64_t)dst_ld * box0.da[d] + box0.db[d];
      if (s < 0 || t < 0 || s >= ((int64_t)1 << 31) || t >= ((int64_t)1 << 31)) ok = false;
      sspan += (int64_t)(box0.dims[d] - 1) * s;
      dspan += (int64_t)(box0.dims[d] - 1) * t;
      f.push(box0.dims[d], (int)s, 0, (int)t, 0);
    }
    if (ok && sspan < ((int64_t)1 << 31) && dspan < ((int64_t)1 << 31)) {
      box = f;
      dst_ld = 1;
      if (!terms.empty()) terms[0].ld = 1;
      sel |= kSelFlat;
    }
  }
  box = simplify(box);
  int64_t total = 1;
  for (int i = 0; i < box.ndim; ++i) total *= box.dims[i];
  if (total >= (int64_t)1 << 31) fail(SYM_ERR_UNSUPPORTED, "block larger than 2^31 elements");
  const int term0 = (int)P.terms.size();
  for (Term& t : terms) t.coef_f = (float)t.coef;
  P.terms.insert(P.terms.end(), terms.begin(), terms.end());
  // transposition check
  const int64_t ld0 = terms.empty() ? 1 : terms[0].ld;
  auto src_stride = [&](int d) { return ld0 * box.sa[d] + box.sb[d]; };
  auto dst_unit = [&](int d) {
    return (int64_t)dst_ld * box.da[d] + box.db[d] == 1;
  };
  const int q = box.ndim - 1;
  int pdim = -1;
  if (!terms.empty() && box.ndim >= 2 && src_stride(q) == 1 && !dst_unit(q) && box.dims[q] >= 16) {
    for (int d = 0; d < q; ++d)
      if (dst_unit(d) && box.dims[d] >= 16) pdim = d;
  }
  if (pdim >= 0) {
    Box t;
    for (int d = 0; d < box.ndim; ++d)
      if (d != pdim && d != q) t.push(box.dims[d], box.sa[d], box.sb[d], box.da[d], box.db[d]);
    t.push(box.dims[pdim], box.sa[pdim], box.sb[pdim], box.da[pdim], box.db[pdim]);
    t.push(box.dims[q], box.sa[q], box.sb[q], box.da[q], box.db[q]);
    int64_t outer = 1;
    for (int d = 0; d < t.ndim - 2; ++d) outer *= t.dims[d];
    const int Pd = t.dims[t.ndim - 2], Qd = t.dims[t.ndim - 1];
    const int64_t per = 1;  // outer indices per item (one 32 x 32 tile)
    for (int tp = 0; tp < Pd; tp += 32)
      for (int tq = 0; tq < Qd; tq += 32)
        for (int64_t o = 0; o < outer; o += per) {
          BoxItem it = make_item(t, dst_off, dst_ld, sel | kSelTile, term0, terms);
          it.start = (int)o;
          it.count = (int)std::min<int64_t>(per, outer - o);
          it.p0 = tp;
          it.q0 = tq;
          P.items.push_back(it);
        }
    return;
  }
  for (int64_t st = 0; st < total; st += kChunk) {
    BoxItem it = make_item(box, dst_off, dst_ld, sel, term0, terms);
    it.start = (int)st;
    it.count = (int)std::min<int64_t>(kChunk, total - st);
    P.items.push_back(it);
  }
}

// Fused recoupling (kSelRecouple): destinations d = 0..n_d-1 that share the
// source blocks s = 0..n_s-1 and the box, destination d receiving
// sum_s coef[d][s] source_s.  srcs/dsts hold (offset, ld) of each side (the
// element at box index t is at off + ld <t, a> + <t, b>).  Returns false
// (nothing emitted) when the box's last dim is not contiguous on both sides
// or the group is too large; the caller then emits per-destination items.
bool emit_recouple(Plan& P, const Box& box0, const std::vector<std::pair<int64_t, int64_t>>& srcs,
                   const std::vector<std::pair<int64_t, int64_t>>& dsts, const std::vector<double>& coef,
                   int src_slot, int dst_slot) {
  const int ns = (int)srcs.size(), nd = (int)dsts.size();
  if (ns < 1 || nd < 1 || ns > kMaxRecouple || nd > kMaxRecouple) return false;
  // Walk the destination in memory order (dims by destination stride, ld
  // multiplier first; the last dim is contiguous on both sides and stays
  // last), so that an item writes whole runs of the destination: a 32-byte
  // sector written in parts by items far apart in time is read back from
  // DRAM by the L2 before the rest lands, reading in parts costs no such fill.
  Box box = simplify(box0);
  {
    const int last = box.ndim - 1;
    std::vector<int> ord(last);
    for (int i = 0; i < last; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return box.da[x] != box.da[y] ? box.da[x] > box.da[y] : box.db[x] > box.db[y];
    });
    Box r;
    for (int i : ord) r.push(box.dims[i], box.sa[i], box.sb[i], box.da[i], box.db[i]);
    r.push(box.dims[last], box.sa[last], box.sb[last], box.da[last], box.db[last]);
    box = simplify(r);
  }
  const int q = box.ndim - 1;
  for (auto& x : srcs)
    if (x.second * box.sa[q] + box.sb[q] != 1 || x.second >= ((int64_t)1 << 31)) return false;
  for (auto& x : dsts)
    if (x.second * box.da[q] + box.db[q] != 1 || x.second >= ((int64_t)1 << 31)) return false;
  int64_t total = 1;
  for (int i = 0; i < box.ndim; ++i) total *= box.dims[i];
  if (total >= (int64_t)1 << 31) fail(SYM_ERR_UNSUPPORTED, "block larger than 2^31 elements");
  const int term0 = (int)P.terms.size();
  for (auto& x : srcs) P.terms.push_back(Term{x.first, x.second, 0.0, 0.0f, 0});
  for (auto& x : dsts) P.terms.push_back(Term{x.first, x.second, 0.0, 0.0f, 0});
  for (double c : coef) P.terms.push_back(Term{0, 0, c, (float)c, 0});
  const std::vector<Term> none;
  // items with few sources hold more positions (the kernel walks a lane's
  // positions H = 32 / n_s at a time), so the coefficient staging of an item
  // is shared by about four rounds of loads whatever n_s is
  const int64_t chunk = ns <= 2 ? 4 * kChunk : ns <= 4 ? 2 * kChunk : kChunk;
  for (int64_t st = 0; st < total; st += chunk) {
    BoxItem it = make_item(box, 0, 0, src_slot | (dst_slot << 4) | kSelRecouple, term0, none);
    it.nterm = ns;
    it.p0 = nd;
    it.start = (int)st;
    it.count = (int)std::min<int64_t>(chunk, total - st);
    P.items.push_back(it);
  }
  return true;
}

// A launch of few items (small tensors) splits its fused recoupling items of
// more than kChunk positions back into kChunk-position ones: more items keep
// more warps busy, while a large launch keeps the long items, which share
// one staging of their coefficients over several rounds of loads.
constexpr int kFewItems = 4096;
void split_few_recouple_items(Plan& P, int begin) {
  const int end = (int)P.items.size();
  if (end - begin >= kFewItems) return;
  std::vector<BoxItem> out;
  out.reserve(end - begin);
  for (int i = begin; i < end; ++i) {
    const BoxItem& it = P.items[i];
    if (!(it.sel & kSelRecouple) || it.count <= kChunk) {
      out.push_back(it);
      continue;
    }
    for (int st = 0; st < it.count; st += kChunk) {
      BoxItem c = it;
      c.start = it.start + st;
      c.count = std::min(kChunk, it.count - st);
      out.push_back(c);
    }
  }
  P.items.resize(begin);
  P.items.insert(P.items.end(), out.begin(), out.end());
}

// Fused recoupling of one gather, scatter or permute (SU(2)): destinations
// whose recoupling sums run over the same source sectors (the same leg
// spins) and that write the same buffer form one group, emitted as fused
// items; `done` (sized ndst by the caller) marks the destinations emitted
// that way.  dst_of(d) gives the destination's (offset, ld) and slot,
// src_of(s) a source's (offset, ld), box_of(d, s) the box every member of
// the group shares (the same leg labels give the same block shape).
using OffLd = std::pair<int64_t, int64_t>;
void fuse_recoupling_items(Plan& P, int64_t ndst, const std::vector<TermList>& X, int src_slot,
                           const std::function<bool(int64_t, OffLd&, int&)>& dst_of,
                           const std::function<OffLd(int64_t)>& src_of,
                           const std::function<Box(int64_t, int64_t)>& box_of, std::vector<char>& done) {
  std::map<std::pair<std::vector<int64_t>, int>, std::vector<int64_t>> groups;
  for (int64_t d = 0; d < ndst; ++d) {
    OffLd o;
    int slot;
    if (X[d].size() < 2 || !dst_of(d, o, slot)) continue;
    std::vector<int64_t> key;
    for (auto& pc : X[d]) key.push_back(pc.first);
    std::sort(key.begin(), key.end());
    groups[{key, slot}].push_back(d);
  }
  for (auto& gr : groups) {
    const std::vector<int64_t>& srcs = gr.first.first;
    const std::vector<int64_t>& ds = gr.second;
    std::vector<OffLd> so, dof;
    for (int64_t sidx : srcs) so.push_back(src_of(sidx));
    std::vector<double> coef(ds.size() * srcs.size(), 0.0);
    for (size_t i = 0; i < ds.size(); ++i) {
      OffLd o;
      int slot;
      dst_of(ds[i], o, slot);
      dof.push_back(o);
      for (auto& pc : X[ds[i]])
        coef[i * srcs.size() + (std::lower_bound(srcs.begin(), srcs.end(), pc.first) - srcs.begin())] += pc.second;
    }
    if (emit_recouple(P, box_of(ds[0], srcs[0]), so, dof, coef, src_slot, gr.first.second))
      for (int64_t d : ds) done[d] = 1;
  }
}

void block_strides(const Tensor& T, int64_t s, int* st) {
  int64_t acc = 1;
  for (int l = T.rank - 1; l >= 0; --l) {
    st[l] = (int)acc;
    acc *= T.dim(s, l);
  }
}

// Swap sign of a fermion-parity block moved by perm (destination leg n = source
// leg perm[n]): the swap tensor is -1 for two odd charges and 1 otherwise, so
// the block gains (-1)^(number of pairs of odd legs whose order perm exchanges).
double z2f_swap_sign(const Tensor& src, const std::vector<int>& perm, const std::vector<int>& srcpos) {
  int odd_pairs = 0;
  const int k = (int)perm.size();
  for (int a = 0; a < k; ++a)
    for (int b = a + 1; b < k; ++b)
      if (perm[a] > perm[b] && src.legs[perm[a]].labels[srcpos[perm[a]]] == 1 &&
          src.legs[perm[b]].labels[srcpos[perm[b]]] == 1)
        ++odd_pairs;
  return (odd_pairs & 1) ? -1.0 : 1.0;
}

// terms[s_dst] = (src sector, coef) with dst leg n = src leg perm[n]
std::vector<TermList> make_xform(const Tensor& src, const std::vector<int>& perm, const Tensor& dst) {
  std::vector<TermList> out(dst.nsec());
  const int k = src.rank;
  if (!su2_like(src.group)) {  // U(1), fermion parity: one source block, coefficient 1 or the swap sign
    std::vector<int> key(k);
    for (int64_t s = 0; s < dst.nsec(); ++s) {
      for (int n = 0; n < k; ++n) key[perm[n]] = dst.p(s, n);
      int64_t ss = src.find(key);
      if (ss < 0) fail(SYM_ERR_ARG, "internal: permuted sector missing");
      out[s].push_back({ss, src.group == SYM_Z2F ? z2f_swap_sign(src, perm, key) : 1.0});
    }
    return out;
  }
  int64_t s = 0;
  while (s < dst.nsec()) {
    int64_t e = s + 1;
    while (e < dst.nsec() && std::equal(dst.pos.begin() + e * k, dst.pos.begin() + (e + 1) * k, dst.pos.begin() + s * k))
      ++e;
    std::vector<int> srcpos(k), spins(k);
    for (int n = 0; n < k; ++n) srcpos[perm[n]] = dst.p(s, n);
    for (int l = 0; l < k; ++l) spins[l] = spin_of(src.group, src.legs[l].labels[srcpos[l]]);
    Gamma g = tree_transform(spins, src.tree, perm, dst.tree);  // the spins' recoupling; charges move along
    std::vector<int64_t> so(g.out_labels.size()), si(g.in_labels.size());
    for (size_t o = 0; o < so.size(); ++o) {
      std::vector<int> key(dst.pos.begin() + s * k, dst.pos.begin() + (s + 1) * k);
      key.insert(key.end(), g.out_labels[o].begin(), g.out_labels[o].end());
      so[o] = dst.find(key);
    }
    for (size_t i = 0; i < si.size(); ++i) {
      std::vector<int> key(srcpos);
      key.insert(key.end(), g.in_labels[i].begin(), g.in_labels[i].end());
      si[i] = src.find(key);
    }
    for (size_t o = 0; o < so.size(); ++o) {
      if (so[o] < 0) fail(SYM_ERR_ARG, "internal: recoupled sector missing");
      for (size_t i = 0; i < si.size(); ++i) {
        double c = g.G[o * si.size() + i];
        if (std::fabs(c) > 1e-13 && si[i] >= 0) out[so[o]].push_back({si[i], c});
      }
    }
    s = e;
  }
  return out;
}

std::vector<TermList> transpose_xform(const std::vector<TermList>& x, int64_t nsrc) {
  std::vector<TermList> t(nsrc);
  for (int64_t s = 0; s < (int64_t)x.size(); ++s)
    for (auto& pc : x[s]) t[pc.first].push_back({s, pc.second});
  return t;
}

// Row/column groups of a tensor in matrix form (legs [rows..., cols...],
// SU(2) tree = comb over rows and comb over cols joined at the root).  A
// group key is the positions of the group's legs plus the spins of its
// subtree's nodes below the subtree top (the top is the sector key x).
std::vector<int> row_key(const Tensor& T, int64_t s, int nr) {
  std::vector<int> k(T.pos.begin() + s * T.rank, T.pos.begin() + s * T.rank + nr);
  if (su2_like(T.group) && nr >= 3) k.insert(k.end(), T.inner_of(s), T.inner_of(s) + (nr - 2));
  return k;
}
std::vector<int> col_key(const Tensor& T, int64_t s, int nr) {
  const int nc = T.rank - nr;
  std::vector<int> k(T.pos.begin() + s * T.rank + nr, T.pos.begin() + (s + 1) * T.rank);
  if (su2_like(T.group) && nc >= 3) {
    const int c0 = nr >= 1 ? nr - 1 : 0;
    k.insert(k.end(), T.inner_of(s) + c0, T.inner_of(s) + c0 + (nc - 2));
  }
  return k;
}

struct MatForm {
  int nr = 0, nc = 0;
  std::vector<int> xs;
  std::map<int, int> xi;
  std::vector<int64_t> rows, cols;
  std::vector<int> sx;
  std::vector<int64_t> r0, c0;
  std::map<std::pair<int, std::vector<int>>, int64_t> rowoff, coloff;
};

MatForm make_matform(const Tensor& T, int nr, const std::function<int(int64_t)>& xkey) {
  MatForm M;
  M.nr = nr;
  M.nc = T.rank - nr;
  std::map<int, std::map<std::vector<int>, int64_t>> rg, cg;
  M.sx.resize(T.nsec());
  std::vector<int> xv(T.nsec());
  for (int64_t s = 0; s < T.nsec(); ++s) {
    int x = xkey(s);
    xv[s] = x;
    int64_t rs = 1, cs = 1;
    for (int l = 0; l < nr; ++l) rs *= T.dim(s, l);
    for (int l = nr; l < T.rank; ++l) cs *= T.dim(s, l);
    rg[x][row_key(T, s, nr)] = rs;
    cg[x][col_key(T, s, nr)] = cs;
  }
  for (auto& kv : rg) {
    M.xi[kv.first] = (int)M.xs.size();
    M.xs.push_back(kv.first);
    int64_t off = 0;
    for (auto& g : kv.second) {
      M.rowoff[{kv.first, g.first}] = off;
      off += g.second;
    }
    M.rows.push_back(off);
    int64_t coff = 0;
    for (auto& g : cg[kv.first]) {
      M.coloff[{kv.first, g.first}] = coff;
      coff += g.second;
    }
    M.cols.push_back(coff);
  }
  M.r0.resize(T.nsec());
  M.c0.resize(T.nsec());
  for (int64_t s = 0; s < T.nsec(); ++s) {
    M.sx[s] = M.xi[xv[s]];
    M.r0[s] = M.rowoff[{xv[s], row_key(T, s, nr)}];
    M.c0[s] = M.coloff[{xv[s], col_key(T, s, nr)}];
  }
  return M;
}

// weights of the legs inside their row group (rw) / column group (cw)
void group_weights(const Tensor& Tm, int64_t s, int nr, int* rw, int* cw) {
  int64_t acc = 1;
  for (int n = nr - 1; n >= 0; --n) {
    rw[n] = (int)acc;
    cw[n] = 0;
    acc *= Tm.dim(s, n);
  }
  acc = 1;
  for (int n = Tm.rank - 1; n >= nr; --n) {
    cw[n] = (int)acc;
    rw[n] = 0;
    acc *= Tm.dim(s, n);
  }
}

int su2_top(const Tensor& T, int64_t s, int nr) {
  int nc = T.rank - nr;
  if (nr == 0 || nc == 0) return 0;
  if (nr == 1) return spin_of(T.group, T.label(s, 0));
  return T.inner_of(s)[nr - 2];
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

Tensor permuted_tensor(const Tensor& T, const std::vector<int>& perm, const Tree& tree, int total) {
  std::vector<Leg> legs;
  for (int p : perm) legs.push_back(T.legs[p]);
  return make_tensor(T.group, legs, total, tree);
}

}  // namespace

bool Plan::f64() const { return precision == SYM_PREC_FP64; }

namespace {
int* g_err_word = nullptr;
std::vector<int*> g_extra_err_words;  // registered by sym_contract_noalloc (static device words)
std::mutex g_err_mu;
}  // namespace

int* device_error_word() {
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_word) {
    cudaError_t e = cudaMalloc(&g_err_word, sizeof(int));
    if (e != cudaSuccess) {
      g_err_word = nullptr;
      fail(SYM_ERR_CUDA, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    cudaMemset(g_err_word, 0, sizeof(int));
  }
  return g_err_word;
}

void register_device_error_word(int* w) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (std::find(g_extra_err_words.begin(), g_extra_err_words.end(), w) == g_extra_err_words.end())
    g_extra_err_words.push_back(w);
}

int take_device_error() {
  std::lock_guard<std::mutex> lk(g_err_mu);
  std::vector<int*> words = g_extra_err_words;
  if (g_err_word) words.insert(words.begin(), g_err_word);
  int code = SYM_OK;
  for (int* w : words) {
    int h = 0;
    if (cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SYM_ERR_CUDA;
    if (h != 0) {
      cudaMemset(w, 0, sizeof(int));
      if (code == SYM_OK) code = h;
    }
  }
  return code;
}

void* DeviceArena::alloc(size_t bytes, bool zero) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? SYM_ERR_OOM : SYM_ERR_CUDA,
         std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  ptrs.push_back(p);
  if (zero) {
    e = cudaMemset(p, 0, bytes);
    if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaMemset failed: ") + cudaGetErrorString(e));
  }
  return p;
}

DeviceArena::~DeviceArena() {
  for (void* p : ptrs) cudaFree(p);
}

// Largest element offset every box item can touch, checked against the size
// of the buffer in its source / destination slot (elements).  Strides are
// non-negative, so the extreme is at the last index of every dimension.
void Plan::validate(const int64_t* src_elems, const int64_t* dst_elems) const {
  for (const BoxItem& it : items) {
    if (it.term0 < 0 || it.nterm < 0 || (size_t)it.term0 + it.nterm > terms.size())
      fail(SYM_ERR_ARG, "internal: term range out of bounds");
    if (it.ndim < 1 || it.ndim > kMaxDim || it.count <= 0 || it.start < 0) fail(SYM_ERR_ARG, "internal: bad box");
    int64_t sa = 0, sb = 0, da = 0, db = 0, total = 1;
    for (int d = 0; d < it.ndim; ++d) {
      if (it.dims[d] < 1 || it.sa[d] < 0 || it.sb[d] < 0 || it.da[d] < 0 || it.db[d] < 0)
        fail(SYM_ERR_ARG, "internal: negative stride or empty dim in a work item");
      sa += (int64_t)(it.dims[d] - 1) * it.sa[d];
      sb += (int64_t)(it.dims[d] - 1) * it.sb[d];
      da += (int64_t)(it.dims[d] - 1) * it.da[d];
      db += (int64_t)(it.dims[d] - 1) * it.db[d];
      total *= it.dims[d];
      uint32_t m;
      int8_t sh;
      div_magic(it.dims[d], m, sh);
      if (m != it.mag[d] || sh != it.shf[d]) fail(SYM_ERR_ARG, "internal: stale division constants in a work item");
    }
    if (sa >= ((int64_t)1 << 31) || sb >= ((int64_t)1 << 31) || da >= ((int64_t)1 << 31) ||
        db >= ((int64_t)1 << 31))
      fail(SYM_ERR_UNSUPPORTED, "internal: box offsets beyond 32 bits");
    for (int d = it.ndim; d < kMaxDim; ++d) {
      uint32_t m;
      int8_t sh;
      div_magic(1, m, sh);
      if (it.dims[d] != 1 || it.sa[d] || it.sb[d] || it.da[d] || it.db[d] || it.mag[d] != m || it.shf[d] != sh)
        fail(SYM_ERR_ARG, "internal: unused dim of a work item is not a unit dim");
    }
    if ((it.sel & kSelUnit) && (it.nterm != 1 || it.t0_coef != 1.0 || it.t0_coef_f != 1.0f))
      fail(SYM_ERR_ARG, "internal: unit flag on a work item whose coefficient is not 1");
    if (it.sel & kSelFlat) {
      if (it.nterm > 1 || it.dst_ld != 1 || (it.nterm == 1 && (it.t0_ld != 1 || terms[it.term0].ld != 1)))
        fail(SYM_ERR_ARG, "internal: flat work item with a two-part offset");
      for (int d = 0; d < it.ndim; ++d)
        if (it.sb[d] != 0 || it.db[d] != 0) fail(SYM_ERR_ARG, "internal: flat work item with a two-part offset");
    }
    if (it.sel & kSelTile) {
      if (it.ndim < 2) fail(SYM_ERR_ARG, "internal: tile item needs two dims");
      const int64_t outer = total / ((int64_t)it.dims[it.ndim - 2] * it.dims[it.ndim - 1]);
      if ((int64_t)it.start + it.count > outer || it.p0 < 0 || it.q0 < 0 || it.p0 >= it.dims[it.ndim - 2] ||
          it.q0 >= it.dims[it.ndim - 1])
        fail(SYM_ERR_ARG, "internal: tile past its box");
    } else if ((int64_t)it.start + it.count > total) {
      fail(SYM_ERR_ARG, "internal: chunk past its box");
    }
    const int ss = it.sel & 3, ds = (it.sel >> 4) & 7;
    if (ds >= DST_COUNT) fail(SYM_ERR_ARG, "internal: bad destination slot");
    for (int i = 0; i < it.nterm; ++i) {
      const Term& t = terms[it.term0 + i];
      if (t.off < 0 || t.ld < 0 || t.off + t.ld * sa + sb >= src_elems[ss])
        fail(SYM_ERR_ARG, "internal: work item reads past its source buffer");
    }
    if (it.sel & kSelRecouple) {
      const int ns = it.nterm, nd = it.p0;
      if (ns < 1 || nd < 1 || ns > kMaxRecouple || nd > kMaxRecouple || (it.sel & (kSelTile | kSelFlat)) ||
          (size_t)it.term0 + ns + nd + (size_t)ns * nd > terms.size())
        fail(SYM_ERR_ARG, "internal: bad recoupling item");
      for (int i = 0; i < nd; ++i) {
        const Term& t = terms[it.term0 + ns + i];
        if (t.off < 0 || t.ld < 0 || t.off + t.ld * da + db >= dst_elems[ds])
          fail(SYM_ERR_ARG, "internal: recoupling item writes past its destination");
      }
      continue;
    }
    const int64_t last = it.dst_off + (int64_t)it.dst_ld * da + db;
    if (it.dst_off < 0 || last >= dst_elems[ds]) fail(SYM_ERR_ARG, "internal: work item writes past its destination");
  }
}

void Plan::set_item_bytes(Range r, int es_src, int es_dst) {
  if (item_bytes_prefix.size() != items.size() + 1) item_bytes_prefix.assign(items.size() + 1, 0.0);
  for (int i = r.first; i < r.first + r.count; ++i) {
    const BoxItem& it = items[i];
    double elems = (double)it.count;
    if (it.sel & kSelTile)
      elems *= (double)std::min(32, it.dims[it.ndim - 2] - it.p0) * std::min(32, it.dims[it.ndim - 1] - it.q0);
    if (it.sel & kSelRecouple)  // every source read once, every destination written once
      item_bytes_prefix[i + 1] = elems * ((double)it.nterm * es_src + (double)it.p0 * es_dst);
    else
      item_bytes_prefix[i + 1] = elems * ((it.nterm > 0 ? es_src : 0) + es_dst);
  }
}

void Plan::clear_profile() {
  for (auto& p : prof) {
    for (auto& e : p.events) {
      cudaEventDestroy(static_cast<cudaEvent_t>(e.e0));
      cudaEventDestroy(static_cast<cudaEvent_t>(e.e1));
    }
    p = PhaseProfile{};
  }
}

Plan::~Plan() {
  clear_profile();
  for (int i = 0; i < kGemmKinds - 1; ++i) {
    if (side[i]) cudaStreamDestroy(static_cast<cudaStream_t>(side[i]));
    if (ev_join[i]) cudaEventDestroy(static_cast<cudaEvent_t>(ev_join[i]));
  }
  if (ev_fork) cudaEventDestroy(static_cast<cudaEvent_t>(ev_fork));
}

void Plan::encode_maps(const void* img_base) {
  if (maps_base == img_base && maps.size() == tc_ops.size()) return;
  maps.assign(tc_ops.size(), TensorMap{});
  for (size_t i = 0; i < tc_ops.size(); ++i)
    if (int e = encode_operand_map(&maps[i], img_base, tc_ops[i], img_elems))
      fail(SYM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(e) + ") for a tensor-core operand");
  maps_base = img_base;
}

void Plan::upload(bool device) {
  // finish the statistics tables (prefix sums)
  if (item_bytes_prefix.size() != items.size() + 1) item_bytes_prefix.assign(items.size() + 1, 0.0);
  for (size_t i = 0; i < items.size(); ++i) item_bytes_prefix[i + 1] += item_bytes_prefix[i];
  flat_prefix.assign(items.size() + 1, 0);
  recouple_prefix.assign(items.size() + 1, 0);
  for (size_t i = 0; i < items.size(); ++i) {
    flat_prefix[i + 1] = flat_prefix[i] + ((items[i].sel & (kSelFlat | kSelTile)) == kSelFlat ? 1 : 0);
    recouple_prefix[i + 1] = recouple_prefix[i] + ((items[i].sel & kSelRecouple) ? 1 : 0);
  }
  tile_flops_prefix.assign(tiles.size() + 1, 0.0);
  tile_bytes_prefix.assign(tiles.size() + 1, 0.0);
  for (size_t i = 0; i < tiles.size(); ++i) {
    const GemmTile& t = tiles[i];
    int64_t m, n, TM, TN;
    if (tile_kind[i] == 0) {
      m = secs_tc[t.sector].m;
      n = secs_tc[t.sector].n;
      TM = TN = 128;
    } else {
      m = secs_simt[t.sector].m;
      n = secs_simt[t.sector].n;
      const int kd = tile_kind[i];
      TM = kd == 1 ? 64 : kd == 2 ? 256 : kd == 3 ? 8 : 256;
      TN = kd == 1 ? 64 : kd == 2 ? 16 : kd == 3 ? 8 : 16;
    }
    double fl;
    const int64_t k = tile_kind[i] == 0 ? secs_tc[t.sector].k : secs_simt[t.sector].k;
    if (tile_kind[i] == 4) {  // rows: [k0, k1) are rows, the reduction is whole
      fl = 2.0 * (double)(t.k1 - t.k0) * (double)n * (double)k;
    } else {
      const int64_t r = std::min<int64_t>(TM, m - t.mt * TM), c = std::min<int64_t>(TN, n - t.nt * TN);
      fl = 2.0 * (double)r * (double)c * (double)(t.k1 - t.k0);
    }
    tile_flops_prefix[i + 1] = tile_flops_prefix[i] + fl;
    // algorithmic bytes: the sector's A, B and C once, shared out by flops
    const double es = f64() ? 8.0 : 4.0;
    const double sector_bytes = es * ((double)m * k + (double)k * n + (double)m * n);
    tile_bytes_prefix[i + 1] = tile_bytes_prefix[i] + sector_bytes * fl / (2.0 * (double)m * n * k);
  }
  // direct items: algorithmic bytes (every column read or written once per
  // position) and useful flops (2 ns nd per position)
  ditem_bytes_prefix.assign(ditems.size() + 1, 0.0);
  ditem_flops_prefix.assign(ditems.size() + 1, 0.0);
  {
    const double es = f64() ? 8.0 : 4.0;
    for (size_t i = 0; i < ditems.size(); ++i) {
      const DirectItem& it = ditems[i];
      ditem_bytes_prefix[i + 1] = ditem_bytes_prefix[i] + (double)it.count * (it.ns + it.nd) * es;
      ditem_flops_prefix[i + 1] = ditem_flops_prefix[i] + 2.0 * (double)it.count * it.ns * it.nd;
    }
  }
  const char* dry_env = std::getenv("SYM_PLAN_DRYRUN");
  if (!device || (dry_env && dry_env[0] == '1')) {
    dry = true;  // host-only planning and validation; the plan cannot run
    return;
  }
  auto up = [&](const void* h, size_t bytes) -> void* {
    void* d = arena.alloc(bytes, false);
    if (bytes) {
      cudaError_t e = cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("cudaMemcpy failed: ") + cudaGetErrorString(e));
    }
    return d;
  };
  d_items = static_cast<BoxItem*>(up(items.data(), items.size() * sizeof(BoxItem)));
  d_terms = static_cast<Term*>(up(terms.data(), terms.size() * sizeof(Term)));
  d_secs_simt = static_cast<GemmSectorSimt*>(up(secs_simt.data(), secs_simt.size() * sizeof(GemmSectorSimt)));
  d_secs_tc = static_cast<TcSector*>(up(secs_tc.data(), secs_tc.size() * sizeof(TcSector)));
  d_tiles = static_cast<GemmTile*>(up(tiles.data(), tiles.size() * sizeof(GemmTile)));
  d_ditems = static_cast<DirectItem*>(up(ditems.data(), ditems.size() * sizeof(DirectItem)));
  if (kind == CONTRACT) {
    const size_t es = f64() ? sizeof(double) : sizeof(float);
    if (img_elems > 0) {  // hi and lo planes; the TMA loads fill past-the-edge boxes with zeros
      img = arena.alloc(img_elems * 2 * 2, false);
      encode_maps(img);
      d_maps = static_cast<TensorMap*>(up(maps.data(), maps.size() * sizeof(TensorMap)));
    }
    lin = arena.alloc(lin_elems * es, false);
    outm = arena.alloc(outm_elems * es, false);
  }
  d_err = device_error_word();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e));
}

// fused charge of two abelian labels (U(1): sum; fermion parity: sum mod 2)
int abelian_fuse(int group, int a, int b) { return group == SYM_Z2F ? (a ^ b) : a + b; }

// Label of the leg fused from labels a and b: U(1), fermion parity as above;
// SU(2): the node spin s of the pair; SU(2) x U(1): the charges' sum with s.
int fused_pair_label(int group, int a, int b, int s) {
  if (group == SYM_SU2) return s;
  if (group == SYM_SU2U1) return su2u1_label(charge_of(group, a) + charge_of(group, b), s);
  return abelian_fuse(group, a, b);
}
bool z2f_group(int group) { return group == SYM_Z2F; }

Leg fused_leg(const Leg& a, const Leg& b, int group) {
  if (a.dir != b.dir) fail(SYM_ERR_INCOMPATIBLE_LEGS, "fused legs must have equal directions");
  std::map<int, int64_t> deg;
  for (size_t i = 0; i < a.labels.size(); ++i)
    for (size_t j = 0; j < b.labels.size(); ++j) {
      int64_t d = (int64_t)a.degens[i] * b.degens[j];
      if (group == SYM_U1) {
        deg[a.labels[i] + b.labels[j]] += d;
      } else if (group == SYM_Z2F) {
        deg[a.labels[i] ^ b.labels[j]] += d;
      } else if (group == SYM_SU2U1) {  // charges add, spins couple
        const int ja = spin_of(group, a.labels[i]), jb = spin_of(group, b.labels[j]);
        const int q = charge_of(group, a.labels[i]) + charge_of(group, b.labels[j]);
        for (int c = std::abs(ja - jb); c <= ja + jb; c += 2) deg[su2u1_label(q, c)] += d;
      } else {
        for (int c = std::abs(a.labels[i] - b.labels[j]); c <= a.labels[i] + b.labels[j]; c += 2) deg[c] += d;
      }
    }
  Leg d;
  d.dir = a.dir;
  for (auto& kv : deg) {
    if (kv.second >= (int64_t)1 << 31) fail(SYM_ERR_UNSUPPORTED, "fused degeneracy too large");
    d.labels.push_back(kv.first);
    d.degens.push_back((int)kv.second);
  }
  return d;
}

// offset of the pair (ia, ib) inside fused label c (pairs: ia slowest)
static int64_t pair_offset(const Leg& a, const Leg& b, int group, int c, int ia, int ib) {
  int64_t off = 0;
  for (size_t i = 0; i < a.labels.size(); ++i)
    for (size_t j = 0; j < b.labels.size(); ++j) {
      bool ok = group == SYM_U1    ? a.labels[i] + b.labels[j] == c
                : group == SYM_Z2F ? (a.labels[i] ^ b.labels[j]) == c
                : group == SYM_SU2U1
                    ? charge_of(group, a.labels[i]) + charge_of(group, b.labels[j]) == charge_of(group, c) &&
                          triangle(spin_of(group, a.labels[i]), spin_of(group, b.labels[j]), spin_of(group, c))
                    : triangle(a.labels[i], b.labels[j], c);
      if (!ok) continue;
      if ((int)i == ia && (int)j == ib) return off;
      off += (int64_t)a.degens[i] * b.degens[j];
    }
  fail(SYM_ERR_ARG, "internal: pair not in fused label");
}

Tree fuse_pair_tree(int k, int f) {
  Tree t;
  t.k = k;
  t.nodes.push_back({f, f + 1});
  std::vector<int> items;
  for (int i = 0; i < k; ++i) {
    if (i == f) items.push_back(k);
    else if (i != f + 1) items.push_back(i);
  }
  int top = items[0];
  for (size_t i = 1; i < items.size(); ++i) {
    t.nodes.push_back({top, items[i]});
    top = k + (int)t.nodes.size() - 1;
  }
  t.validate();
  return t;
}

// ------------------------------------------------------------------ transforms --
// mode 0: permute (out leg n = in leg perm[n]); 1: fuse legs (leg, leg+1);
// 2: split leg `leg` of `in` into out legs (leg, leg+1).
std::unique_ptr<Plan> plan_transform(const Tensor& in, const Tensor& out, const std::vector<int>& perm,
                                     int precision, int mode, int leg) {
  auto P = std::make_unique<Plan>();
  P->kind = Plan::TRANSFORM;
  P->precision = precision;
  P->numel_a = in.numel();
  P->numel_c = out.numel();
  const int k = in.rank;
  int ist[kMaxDim], ost[kMaxDim];
  if (mode == 0) {
    std::vector<int> pinv(k);
    for (int n = 0; n < k; ++n) pinv[perm[n]] = n;
    auto X = make_xform(in, perm, out);
    std::vector<char> done(out.nsec(), 0);
    if (su2_like(in.group))  // output labels sharing their sources: one fused item per position range
      fuse_recoupling_items(
          *P, out.nsec(), X, 0,
          [&](int64_t s, OffLd& o, int& slot) {
            o = {out.offs[s], 1};
            slot = DST_OUT;
            return true;
          },
          [&](int64_t si) { return OffLd{in.offs[si], 1}; },
          [&](int64_t s, int64_t si) {
            block_strides(out, s, ost);
            block_strides(in, si, ist);
            Box b;
            for (int l = 0; l < k; ++l) b.push(out.dim(s, pinv[l]), ist[l], 0, ost[pinv[l]], 0);
            return b;
          },
          done);
    for (int64_t s = 0; s < out.nsec(); ++s) {
      if (done[s]) continue;
      block_strides(out, s, ost);
      std::vector<Term> terms;
      for (auto& pc : X[s]) terms.push_back({in.offs[pc.first], 1, pc.second});
      Box b;
      int64_t src0 = X[s].empty() ? -1 : X[s][0].first;
      for (int l = 0; l < k; ++l) {
        int d = out.dim(s, pinv[l]);
        int sst = 0;
        if (src0 >= 0) {
          block_strides(in, src0, ist);
          sst = ist[l];
        }
        b.push(d, sst, 0, ost[pinv[l]], 0);
      }
      emit(*P, b, out.offs[s], 1, 0, DST_OUT, terms);
    }
  } else if (mode == 1) {
    const int f = leg;
    const Leg& la = in.legs[f];
    const Leg& lb = in.legs[f + 1];
    const Leg& ld = out.legs[f];
    const bool tree = su2_like(in.group);
    Tensor mid = tree ? make_tensor(in.group, in.legs, in.total, fuse_pair_tree(k, f)) : in;
    std::vector<TermList> X;
    std::vector<int> idp(k);
    for (int i = 0; i < k; ++i) idp[i] = i;
    if (tree) X = make_xform(in, idp, mid);
    // out sector of mid sector sm and the row of the fused leg where it starts
    auto place = [&](int64_t sm, int64_t& row0) {
      int c = fused_pair_label(in.group, la.labels[mid.p(sm, f)], lb.labels[mid.p(sm, f + 1)],
                               tree ? mid.inner_of(sm)[0] : 0);
      int iq = (int)(std::lower_bound(ld.labels.begin(), ld.labels.end(), c) - ld.labels.begin());
      std::vector<int> key;
      for (int l = 0; l < k; ++l) {
        if (l == f) key.push_back(iq);
        else if (l != f + 1) key.push_back(mid.p(sm, l));
      }
      if (tree) key.insert(key.end(), mid.inner_of(sm) + 1, mid.inner_of(sm) + mid.nin);
      int64_t so = out.find(key);
      if (so < 0) fail(SYM_ERR_ARG, "internal: fused sector missing");
      row0 = pair_offset(la, lb, in.group, c, mid.p(sm, f), mid.p(sm, f + 1));
      return so;
    };
    std::vector<char> done(mid.nsec(), 0);
    if (tree)  // the mid sectors of one set of leg labels differ in the fused leg's label, so
               // in its dimension D: out strides of legs before f are D x (strides without it),
               // taken as the destination's ld
      fuse_recoupling_items(
          *P, mid.nsec(), X, 0,
          [&](int64_t sm, OffLd& o, int& slot) {
            int64_t row0;
            const int64_t so = place(sm, row0);
            block_strides(out, so, ost);
            o = {out.offs[so] + row0 * ost[f], out.dim(so, f)};
            slot = DST_OUT;
            return true;
          },
          [&](int64_t si) { return OffLd{in.offs[si], 1}; },
          [&](int64_t sm, int64_t si) {
            int64_t row0;
            const int64_t so = place(sm, row0);
            block_strides(out, so, ost);
            block_strides(in, si, ist);
            const int D = out.dim(so, f), db_ = mid.dim(sm, f + 1);
            Box b;
            for (int l = 0; l < k; ++l) {
              const int d = mid.dim(sm, l);
              if (l < f) {
                if (ost[l] % D != 0) fail(SYM_ERR_ARG, "internal: fused leg's dimension does not divide a stride");
                b.push(d, ist[l], 0, ost[l] / D, 0);
              } else {
                b.push(d, ist[l], 0, 0, l == f ? db_ * ost[f] : l == f + 1 ? ost[f] : ost[l - 1]);
              }
            }
            return b;
          },
          done);
    for (int64_t sm = 0; sm < mid.nsec(); ++sm) {
      if (done[sm]) continue;
      int64_t row0;
      const int64_t so = place(sm, row0);
      block_strides(out, so, ost);
      std::vector<Term> terms;
      if (!tree) {
        terms.push_back({in.offs[sm], 1, 1.0});
      } else {
        for (auto& pc : X[sm]) terms.push_back({in.offs[pc.first], 1, pc.second});
      }
      block_strides(in, !tree ? sm : (X[sm].empty() ? 0 : X[sm][0].first), ist);
      Box b;
      int db_ = mid.dim(sm, f + 1);
      for (int l = 0; l < k; ++l) {
        int d = mid.dim(sm, l);
        int dst = l < f ? ost[l] : l == f ? db_ * ost[f] : l == f + 1 ? ost[f] : ost[l - 1];
        b.push(d, ist[l], 0, dst, 0);
      }
      emit(*P, b, out.offs[so] + row0 * ost[f], 1, 0, DST_OUT, terms);
    }
  } else {
    const int f = leg;  // out legs f, f+1 come from in leg f
    const int ko = out.rank;
    const Leg& la = out.legs[f];
    const Leg& lb = out.legs[f + 1];
    const bool tree = su2_like(in.group);
    Tensor mid = tree ? make_tensor(in.group, out.legs, in.total, fuse_pair_tree(ko, f)) : out;
    std::vector<TermList> X;
    std::vector<int> idp(ko);
    for (int i = 0; i < ko; ++i) idp[i] = i;
    if (tree) X = make_xform(mid, idp, out);
    // where each mid sector lives inside `in`
    std::vector<int64_t> m_in(mid.nsec()), m_row(mid.nsec());
    for (int64_t sm = 0; sm < mid.nsec(); ++sm) {
      int c = fused_pair_label(in.group, la.labels[mid.p(sm, f)], lb.labels[mid.p(sm, f + 1)],
                               tree ? mid.inner_of(sm)[0] : 0);
      const Leg& lf = in.legs[f];
      int iq = (int)(std::lower_bound(lf.labels.begin(), lf.labels.end(), c) - lf.labels.begin());
      std::vector<int> key;
      for (int l = 0; l < ko; ++l) {
        if (l == f) key.push_back(iq);
        else if (l != f + 1) key.push_back(mid.p(sm, l));
      }
      if (tree) key.insert(key.end(), mid.inner_of(sm) + 1, mid.inner_of(sm) + mid.nin);
      m_in[sm] = in.find(key);
      if (m_in[sm] < 0) fail(SYM_ERR_ARG, "internal: split source sector missing");
      m_row[sm] = pair_offset(la, lb, in.group, c, mid.p(sm, f), mid.p(sm, f + 1));
    }
    // source box of mid sector sm (the fused leg f of `in` seen as legs f, f+1)
    auto src_box = [&](int64_t sm, int* sa_, int* sb_) {
      const int64_t si = m_in[sm];
      block_strides(in, si, ist);
      const int64_t dfused = in.dim(si, f);
      const int stf = ist[f];
      for (int l = 0; l < f; ++l) {  // in legs l < f: stride = dfused * (stride without the fused dim)
        sa_[l] = (int)(ist[l] / dfused);
        sb_[l] = 0;
      }
      sa_[f] = 0;
      sb_[f] = (int)(mid.dim(sm, f + 1) * stf);
      sa_[f + 1] = 0;
      sb_[f + 1] = stf;
      for (int l = f + 2; l < ko; ++l) {
        sa_[l] = 0;
        sb_[l] = ist[l - 1];
      }
      return OffLd{in.offs[si] + m_row[sm] * stf, dfused};
    };
    std::vector<char> done(out.nsec(), 0);
    if (tree)
      fuse_recoupling_items(
          *P, out.nsec(), X, 0,
          [&](int64_t s, OffLd& o, int& slot) {
            o = {out.offs[s], 1};
            slot = DST_OUT;
            return true;
          },
          [&](int64_t sm) {
            int sa_[kMaxDim], sb_[kMaxDim];
            return src_box(sm, sa_, sb_);
          },
          [&](int64_t s, int64_t sm) {
            int sa_[kMaxDim], sb_[kMaxDim];
            src_box(sm, sa_, sb_);
            block_strides(out, s, ost);
            Box b;
            for (int l = 0; l < ko; ++l) b.push(out.dim(s, l), sa_[l], sb_[l], ost[l], 0);
            return b;
          },
          done);
    for (int64_t s = 0; s < out.nsec(); ++s) {
      if (done[s]) continue;
      block_strides(out, s, ost);
      TermList tl = !tree ? TermList{{s, 1.0}} : X[s];
      std::vector<Term> terms;
      int sa_[kMaxDim] = {0}, sb_[kMaxDim] = {0};
      bool first = true;
      for (auto& pc : tl) {
        int64_t sm = pc.first;
        int64_t si = m_in[sm];
        block_strides(in, si, ist);
        int64_t dfused = in.dim(si, f);
        int64_t stf = ist[f];
        terms.push_back({in.offs[si] + m_row[sm] * stf, dfused, pc.second});
        if (first) {
          // in legs l < f: stride = dfused * (stride without the fused dim)
          for (int l = 0; l < f; ++l) {
            sa_[l] = (int)(ist[l] / dfused);
            sb_[l] = 0;
          }
          sa_[f] = 0;
          sb_[f] = (int)(mid.dim(sm, f + 1) * stf);
          sa_[f + 1] = 0;
          sb_[f + 1] = (int)stf;
          for (int l = f + 2; l < ko; ++l) {
            sa_[l] = 0;
            sb_[l] = ist[l - 1];
          }
          first = false;
        }
      }
      Box b;
      for (int l = 0; l < ko; ++l) b.push(out.dim(s, l), sa_[l], sb_[l], ost[l], 0);
      emit(*P, b, out.offs[s], 1, 0, DST_OUT, terms);
    }
  }
  split_few_recouple_items(*P, 0);
  P->xform = {0, (int)P->items.size()};
  {
    const int es = precision == SYM_PREC_FP64 ? 8 : 4;
    P->set_item_bytes(P->xform, es, es);
  }
  {
    const int64_t src[4] = {in.numel(), 0, 0, 0};
    const int64_t dst[DST_COUNT] = {out.numel(), 0, 0, 0, 0, 0};
    P->validate(src, dst);
  }
  P->upload();
  return P;
}

// ----------------------------------------------------------------- contraction --
namespace {

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

// ------------------------------------------------------ planning parameters --
// Read by every plan built afterwards (plans already built keep theirs).
// Defaults, then SYM_* environment variables, then sym_tune_set.
namespace {
std::mutex tune_mu;
int tune_ver = 0;
sym_tune& tune_state() {
  static sym_tune t = [] {
    sym_tune d;
    d.tc_min_mn = env_int("SYM_TC_MIN_MN", 64);
    d.tc_min_k = env_int("SYM_TC_MIN_K", 48);
    d.tc_max_k = env_int("SYM_TC_MAX_K", 16384);
    d.direct_max = std::max(0, std::min(env_int("SYM_DIRECT_MAX", kMaxDirect), kMaxDirect));
    d.direct_chunk = kDirectApplyChunk;
    d.rows_spans = kRowsSpansPerTile;
    d.splitk_ctas = 2;
    d.thin_slice = 4096;
    d.tc_order = 0;
    d.tc_group = 8;
    d.direct_mixed = 1;
    d.tc_all = 0;
    // SYM_TUNE="name=value,...": any parameter (names as in sym_tune)
    if (const char* e = std::getenv("SYM_TUNE")) {
      std::string all(e);
      size_t p = 0;
      while (p < all.size()) {
        size_t q = all.find(',', p);
        if (q == std::string::npos) q = all.size();
        const std::string kv = all.substr(p, q - p);
        const size_t eq = kv.find('=');
        if (eq != std::string::npos) {
          const std::string k = kv.substr(0, eq);
          const int v = std::atoi(kv.c_str() + eq + 1);
          int* f = k == "tc_min_mn" ? &d.tc_min_mn : k == "tc_min_k" ? &d.tc_min_k : k == "tc_max_k" ? &d.tc_max_k
                 : k == "direct_max" ? &d.direct_max : k == "direct_chunk" ? &d.direct_chunk
                 : k == "rows_spans" ? &d.rows_spans : k == "splitk_ctas" ? &d.splitk_ctas
                 : k == "thin_slice" ? &d.thin_slice : k == "tc_order" ? &d.tc_order
                 : k == "tc_group" ? &d.tc_group : k == "direct_mixed" ? &d.direct_mixed
                 : k == "tc_all" ? &d.tc_all : nullptr;
          if (f) *f = v;
        }
        p = q + 1;
      }
    }
    return d;
  }();
  return t;
}
}  // namespace

sym_tune current_tune() {
  std::lock_guard<std::mutex> g(tune_mu);
  return tune_state();
}

void set_tune(const sym_tune& t) {
  auto in = [](int v, int lo, int hi) { return v >= lo && v <= hi; };
  if (!in(t.tc_min_mn, 1, 1 << 30) || !in(t.tc_min_k, 1, 1 << 30) || !in(t.tc_max_k, t.tc_min_k, 1 << 30) ||
      !in(t.direct_max, 0, kMaxDirect) || !in(t.direct_chunk, 32, 1 << 16) || t.direct_chunk % 32 ||
      !in(t.rows_spans, 1, 64) || !in(t.splitk_ctas, 0, 64) || !in(t.thin_slice, 256, 1 << 20) ||
      t.thin_slice % 256 || !in(t.tc_order, 0, 1) || !in(t.tc_group, 0, 256) || !in(t.direct_mixed, 0, 1) ||
      !in(t.tc_all, 0, 1))
    fail(SYM_ERR_ARG, "planning parameter out of range");
  std::lock_guard<std::mutex> g(tune_mu);
  tune_state() = t;
  ++tune_ver;
}

int tune_epoch() {
  std::lock_guard<std::mutex> g(tune_mu);
  return tune_ver;
}

namespace {

// Kernel choice of one GEMM (m x n result, reduction k) of a split-BF16 plan:
// the tensor cores when the 128 x 128 x 64 tile is well filled, the exact
// FP32 CUDA-core kernel otherwise (thin matrices are bandwidth-bound, and
// very long reductions are split across CTAs there).  The thresholds and
// the schedule parameters are the planning parameters below.
int choose_kind(bool f64, int64_t m, int64_t n, int64_t k, const sym_tune& t) {
  if (!f64 && t.tc_all && k <= t.tc_max_k) return 0;  // long reductions keep the split CUDA-core kernels
  if (m <= 8 && n <= 8) return 3;
  if (k <= 16 && n <= 16) return 4;
  const int simt = n <= 16 ? 2 : 1;
  if (f64) return simt;
  if (m >= t.tc_min_mn && n >= t.tc_min_mn && k >= t.tc_min_k && k <= t.tc_max_k) return 0;
  return simt;
}

}  // namespace

// GEMM tiles and tensor-core operands stay inside their buffers (host check)
void validate_gemms(const Plan& P, bool f64) {
  for (size_t i = 0; i < P.tiles.size(); ++i) {
    const GemmTile& t = P.tiles[i];
    if (P.tile_kind[i] != 0) {
      if (t.sector < 0 || t.sector >= (int)P.secs_simt.size()) fail(SYM_ERR_ARG, "internal: bad GEMM sector index");
      const GemmSectorSimt& s = P.secs_simt[t.sector];
      const bool ta = (s.trans & kTransA) != 0, tb = (s.trans & kTransB) != 0;
      const int64_t a_last = ta ? (int64_t)(s.k - 1) * s.lda + s.m - 1 : (int64_t)(s.m - 1) * s.lda + s.k - 1;
      const int64_t b_last = tb ? (int64_t)(s.n - 1) * s.ldb + s.k - 1 : (int64_t)(s.k - 1) * s.ldb + s.n - 1;
      if (s.m < 1 || s.n < 1 || s.k < 1 || (s.trans & ~(kTransA | kTransB)) != 0 || s.a_off < 0 ||
          s.b_off < 0 || s.c_off < 0 || s.a_off + a_last >= P.lin_elems || s.b_off + b_last >= P.lin_elems ||
          s.c_off + (int64_t)(s.m - 1) * s.ldc + s.n - 1 >= P.outm_elems)
        fail(SYM_ERR_ARG, "internal: CUDA-core GEMM sector past its buffers");
      if (P.tile_kind[i] == 4) {  // rows: [k0, k1) rows of dense A and C, B maybe transposed
        if (t.k0 < 0 || t.k1 > s.m || t.k0 >= t.k1 || s.k > 16 || s.n > 16 || s.lda != s.k || s.ldc != s.n || ta)
          fail(SYM_ERR_ARG, "internal: rows GEMM tile out of range");
      } else {
        if (t.k0 < 0 || t.k1 > s.k || t.k0 >= t.k1) fail(SYM_ERR_ARG, "internal: GEMM tile reduction out of range");
        if (P.tile_kind[i] != 3 && s.trans != 0) fail(SYM_ERR_ARG, "internal: transposed operand on a tile kernel");
        if (P.tile_kind[i] == 3 && (s.m > 8 || s.n > 8)) fail(SYM_ERR_ARG, "internal: thin GEMM too wide");
      }
    } else {
      if (t.sector < 0 || t.sector >= (int)P.secs_tc.size()) fail(SYM_ERR_ARG, "internal: bad GEMM sector index");
      const TcSector& s = P.secs_tc[t.sector];
      const int nops = (int)P.tc_ops.size();
      auto fits = [&](int op, int mn, int64_t mnd, int64_t kd) {  // operand of the M (or N) dim mnd
        if (op < 0 || op >= nops) return false;
        const TcOperand& o = P.tc_ops[op];
        return o.mn == mn && (mn ? (o.cols == mnd && o.rows == kd) : (o.rows == mnd && o.cols == kd));
      };
      if (!fits(s.amap, s.a_mn, s.m, s.k) || !fits(s.bmap, s.b_mn, s.n, s.k) || s.ktiles != cdiv(s.k, 64) ||
          t.mt * 128 >= s.m || t.nt * 128 >= s.n || s.c_off < 0 ||
          s.c_off + (int64_t)(s.m - 1) * s.ldc + s.n - 1 >= P.outm_elems || s.ktiles < 1)
        fail(SYM_ERR_ARG, "internal: tcgen05 GEMM tile past its buffers");
    }
  }
  // tcgen05 operands: rows on 128-byte lines inside the hi plane (TMA rules)
  for (const TcOperand& o : P.tc_ops)
    if (f64 || o.off < 0 || o.off % 64 || o.ld % 64 || o.ld < o.cols || o.rows < 1 || o.cols < 1 ||
        (o.mn != 0 && o.mn != 1) || o.off + (int64_t)o.rows * o.ld > P.img_elems)
      fail(SYM_ERR_ARG, "internal: tensor-core operand past its buffer");
}

// Direct items stay inside the tensors they address: numel_a (A, dA),
// numel_b (B, dB), numel_c (C, dC); strides non-negative, so the extreme of
// every column is at the last index of every dim, and each column's span
// stays below 2^31 (the kernel forms it in 32 bits).
void validate_direct(const Plan& P) {
  const int64_t ne[3] = {P.numel_a, P.numel_b, P.numel_c};
  // tensor of a source slot (0 A, 1 B, 2 dC) and of a destination slot
  auto src_space = [](int slot) { return slot == 0 ? 0 : slot == 1 ? 1 : slot == 2 ? 2 : -1; };
  auto dst_space = [](int slot) { return slot == DST_OUT ? 2 : slot == DST_DA ? 0 : slot == DST_DB ? 1 : -1; };
  const Range rs[3] = {P.fwd_direct, P.bwd_direct_a, P.bwd_direct_b};
  int expect = 0;
  for (const Range& r : rs) {
    if (r.first != expect || r.count < 0) fail(SYM_ERR_ARG, "internal: direct ranges out of order");
    expect += r.count;
  }
  if (expect != (int)P.ditems.size()) fail(SYM_ERR_ARG, "internal: direct ranges do not cover the items");
  for (int r = 0; r < 3; ++r)  // every launch runs one item kind
    for (int i = rs[r].first; i < rs[r].first + rs[r].count; ++i)
      if (P.ditems[i].op != (r == 2 ? kDirectOuter : kDirectApply)) fail(SYM_ERR_ARG, "internal: direct item kind");
  for (const DirectItem& it : P.ditems) {
    if ((it.op != kDirectApply && it.op != kDirectOuter) || it.ns < 1 || it.nd < 1 || it.ns > kMaxDirect ||
        it.nd > kMaxDirect || it.ndim < 1 || it.ndim > kDirectDims || it.start < 0 || it.count < 1)
      fail(SYM_ERR_ARG, "internal: bad direct item");
    int64_t total = 1;
    for (int d = 0; d < kDirectDims; ++d) {
      if (it.dims[d] < 1 || (d >= it.ndim && it.dims[d] != 1))
        fail(SYM_ERR_ARG, "internal: bad dim in a direct item");
      uint32_t m;
      int8_t sh;
      div_magic(it.dims[d], m, sh);
      if (m != it.mag[d] || sh != (int8_t)((it.shf >> (8 * d)) & 0xff))
        fail(SYM_ERR_ARG, "internal: stale division constants in a direct item");
      total *= it.dims[d];
    }
    if ((int64_t)it.start + it.count > total) fail(SYM_ERR_ARG, "internal: direct item past its box");
    const int s1 = it.slots & 3, s2 = (it.slots >> 2) & 3, ds = (it.slots >> 4) & 7;
    const int sp = src_space(s1);
    const int qp = it.op == kDirectApply ? dst_space(ds) : src_space(s2);  // space of the d columns
    const int kp = it.op == kDirectApply ? src_space(s2) : dst_space(ds);  // space of the coefficient offsets
    if (sp < 0 || qp < 0 || kp != 1) fail(SYM_ERR_ARG, "internal: bad slot in a direct item");
    auto check = [&](const DirectCol& c, int space) {
      int64_t span = 0;
      for (int d = 0; d < kDirectDims; ++d) {
        if (c.str[d] < 0 || (d >= it.ndim && c.str[d] != 0)) fail(SYM_ERR_ARG, "internal: bad direct column stride");
        span += (int64_t)(it.dims[d] - 1) * c.str[d];
      }
      if (c.off < 0 || span >= ((int64_t)1 << 31) || c.off + span >= ne[space])
        fail(SYM_ERR_ARG, "internal: direct item addresses past its tensor");
    };
    for (int c = 0; c < it.ns; ++c) check(it.src[c], sp);
    for (int c = 0; c < it.nd; ++c) check(it.dst[c], qp);
    for (int e = 0; e < kMaxDirect * kMaxDirect; ++e) {
      const int d = e / kMaxDirect, c = e % kMaxDirect;
      if (it.kc[e] == 0.0) continue;
      if (d >= it.nd || c >= it.ns || it.koff[e] < 0 || it.koff[e] >= ne[kp])
        fail(SYM_ERR_ARG, "internal: direct coefficient past its tensor");
    }
  }
}

std::unique_ptr<Plan> plan_contract(const Tensor& A, const Tensor& B, const std::vector<int>& pairsA,
                                    const std::vector<int>& pairsB, const Tensor& C, int precision, bool device) {
  auto P = std::make_unique<Plan>();
  P->kind = Plan::CONTRACT;
  P->precision = precision;
  const bool f64 = precision == SYM_PREC_FP64;
  const sym_tune tp = current_tune();
  P->tc_order = tp.tc_order;
  const int nc = (int)pairsA.size();
  std::vector<int> freeA, freeB;
  for (int l = 0; l < A.rank; ++l)
    if (std::find(pairsA.begin(), pairsA.end(), l) == pairsA.end()) freeA.push_back(l);
  for (int l = 0; l < B.rank; ++l)
    if (std::find(pairsB.begin(), pairsB.end(), l) == pairsB.end()) freeB.push_back(l);
  const int na = (int)freeA.size(), nb = (int)freeB.size();
  std::vector<int> permA(freeA), permB(pairsB);
  permA.insert(permA.end(), pairsA.begin(), pairsA.end());
  permB.insert(permB.end(), freeB.begin(), freeB.end());
  const bool su2 = su2_like(A.group);  // tree decompositions: SU(2), SU(2) x U(1)
  const bool composite = A.group == SYM_SU2U1;
  Tensor Am = permuted_tensor(A, permA, Tree::comb_pair(na, nc), A.total);
  Tensor Bm = permuted_tensor(B, permB, Tree::comb_pair(nc, nb), B.total);
  std::vector<Leg> clegs;
  for (int l : freeA) clegs.push_back(A.legs[l]);
  for (int l : freeB) clegs.push_back(B.legs[l]);
  Tensor Cn = make_tensor(A.group, clegs, z2f_group(A.group) ? (A.total ^ B.total) : A.total + B.total,
                          Tree::comb_pair(na, nb));
  const bool natural = !su2 || C.tree == Cn.tree;

  auto XA = make_xform(A, permA, Am);
  auto XB = make_xform(B, permB, Bm);
  // SU(2) normalisation folded into A's gather terms
  if (su2) {
    for (int64_t s = 0; s < Am.nsec(); ++s) {
      int x = su2_top(Am, s, na);
      double f = ((x & 1) ? -1.0 : 1.0) / std::sqrt((double)x + 1.0);
      for (int i = 0; i < nc; ++i)
        if (A.legs[pairsA[i]].dir == -1 && (spin_of(A.group, Am.label(s, na + i)) & 1)) f = -f;
      for (auto& pc : XA[s]) pc.second *= f;
    }
  }
  std::vector<TermList> XC, XCt;
  if (!natural) {
    std::vector<int> idp(C.rank);
    for (int i = 0; i < C.rank; ++i) idp[i] = i;
    XC = make_xform(Cn, idp, C);
    XCt = transpose_xform(XC, Cn.nsec());
  }
  auto XAt = transpose_xform(XA, A.nsec());
  auto XBt = transpose_xform(XB, B.nsec());

  // sector key x of the matrix form: SU(2) coupled spin; U(1) charge of the
  // contracted legs as A sees them; fermion parity of the contracted legs;
  // SU(2) x U(1) both, as 4096 q + 2j (a coupled spin of at most six legs
  // below 64 each stays below 4096)
  const bool z2f = A.group == SYM_Z2F;
  auto q_of = [&](const Tensor& T, int64_t s, int n) {
    return composite ? charge_of(T.group, T.label(s, n)) : T.label(s, n);
  };
  auto both = [&](int q, int spin) { return composite ? 4096 * q + spin : spin; };
  auto keyA = [&](int64_t s) {
    int x = 0;
    if (!su2 || composite)
      for (int n = na; n < Am.rank; ++n) x = z2f ? x ^ Am.label(s, n) : x + Am.legs[n].dir * q_of(Am, s, n);
    return su2 ? both(x, su2_top(Am, s, na)) : x;
  };
  auto keyB = [&](int64_t s) {
    int x = 0;
    if (!su2 || composite)
      for (int n = 0; n < nc; ++n) x = z2f ? x ^ Bm.label(s, n) : x - Bm.legs[n].dir * q_of(Bm, s, n);
    return su2 ? both(x, su2_top(Bm, s, nc)) : x;
  };
  auto keyC = [&](int64_t s) {
    int x = su2 && !composite ? 0 : A.total;
    if (!su2 || composite)
      for (int n = 0; n < na; ++n) x = z2f ? x ^ Cn.label(s, n) : x - Cn.legs[n].dir * q_of(Cn, s, n);
    return su2 ? both(x, su2_top(Cn, s, na)) : x;
  };
  MatForm MA = make_matform(Am, na, keyA);
  MatForm MB = make_matform(Bm, nc, keyB);
  MatForm MC = make_matform(Cn, na, keyC);

  // GEMM sectors: x present on both sides.  Per sector three GEMMs:
  // forward C = A B (m n k), dA = dC B^T (m k n), dB = A^T dC (k n m).
  struct G {
    int x;
    int64_t m, n, k;
    int kind[3];
    // linear FP32/FP64 operands of the CUDA-core GEMMs (elements of `lin`):
    // forward A (m x k), B (k x n); dA B^T (n x k); dB A^T (k x m); dC (m x n)
    int64_t a = -1, b = -1, bt = -1, at = -1, dcl = -1;
    // split-BF16 buffers of the tcgen05 GEMMs (elements of the hi plane),
    // stored A (m x k), B (k x n), dC (m x n) and read K-major or MN-major:
    // forward A (K), B (MN); dA dC (K), B (K); dB A (MN), dC (MN).  The
    // forward's A and B serve the backward unchanged.
    int64_t ta = -1, tb = -1, tdc = -1;
    int fa = -1, fb = -1, dAa = -1, dAb = -1, dBa = -1, dBb = -1;  // map indices (P->tc_ops)
    int64_t c, da, db;  // output matrices
    bool split[3];
  };
  std::vector<G> gs;
  std::map<int, int> gofx;
  for (size_t i = 0; i < MA.xs.size(); ++i) {
    auto it = MB.xi.find(MA.xs[i]);
    if (it == MB.xi.end()) continue;
    G g{};
    g.x = MA.xs[i];
    g.m = MA.rows[i];
    g.k = MA.cols[i];
    g.n = MB.cols[it->second];
    if (MB.rows[it->second] != g.k) fail(SYM_ERR_INCOMPATIBLE_LEGS, "contracted sector dimensions differ");
    if (g.m <= 0 || g.n <= 0 || g.k <= 0) continue;
    if (g.m >= ((int64_t)1 << 31) || g.n >= ((int64_t)1 << 31) || g.k >= ((int64_t)1 << 31))
      fail(SYM_ERR_UNSUPPORTED, "sector matrix dimension too large");
    g.kind[0] = choose_kind(f64, g.m, g.n, g.k, tp);
    g.kind[1] = choose_kind(f64, g.m, g.k, g.n, tp);
    g.kind[2] = choose_kind(f64, g.k, g.n, g.m, tp);
    gofx[g.x] = (int)gs.size();
    gs.push_back(g);
  }

  // ---- direct sectors (U(1), B_x at most kMaxDirect x kMaxDirect): the
  // product runs on A's and C's blocks (kernels.h, DirectItem).  Such sectors
  // leave gs: no matrix form, GEMM, gather or scatter of their own (the dB
  // scatter below still zero-fills their dB blocks for the atomic reduction).
  std::set<int> dset;
  std::vector<DirectItem> dfw, dba, dbb;
  int rw[kMaxDim], cw[kMaxDim], st[kMaxDim];
  if (!su2 && C.nsec() == Cn.nsec()) {
    const int dmax = tp.direct_max;
    std::map<int, std::map<std::vector<int>, std::vector<int64_t>>> arow, crow;  // x -> row key -> sectors
    std::map<int, std::vector<int64_t>> bsec;                                   // x -> Bm sectors
    for (int64_t s = 0; s < Am.nsec(); ++s) arow[MA.xs[MA.sx[s]]][row_key(Am, s, na)].push_back(s);
    for (int64_t s = 0; s < Cn.nsec(); ++s) crow[MC.xs[MC.sx[s]]][row_key(Cn, s, na)].push_back(s);
    for (int64_t s = 0; s < Bm.nsec(); ++s) bsec[MB.xs[MB.sx[s]]].push_back(s);
    // one column of a row group: matrix column, offset of the free origin,
    // strides of the free legs in its block
    struct Col {
      int64_t idx, off;
      std::vector<int64_t> fs;
      double sgn = 1.0;  // coefficient of the source block (a fermion-parity swap sign, else 1)
    };
    // enumerate the index tuples of dims[lo..hi) (last fastest)
    auto each = [](const std::vector<int>& dims, int lo, int hi, const std::function<void(const int*)>& fn) {
      std::vector<int> t(dims.size(), 0);
      int64_t tot = 1;
      for (int n = lo; n < hi; ++n) tot *= dims[n];
      for (int64_t e = 0; e < tot; ++e) {
        int64_t r = e;
        for (int n = hi - 1; n >= lo; --n) {
          t[n] = (int)(r % dims[n]);
          r /= dims[n];
        }
        fn(t.data());
      }
    };
    // ld[c], sa[n], sb[n] with fs[c][n] = ld[c] sa[n] + sb[n]: one multiplier
    // per column, the stride of the last (innermost) free leg whose stride
    // varies between columns, covers every varying leg
    auto fit = [](const std::vector<Col>& cols, int nf, std::vector<int64_t>& ld, std::vector<int64_t>& sa,
                  std::vector<int64_t>& sb) {
      ld.assign(cols.size(), 1);
      sa.assign(nf, 0);
      sb.assign(nf, 0);
      int n0 = -1;
      for (int n = 0; n < nf; ++n)
        for (auto& c : cols)
          if (c.fs[n] != cols[0].fs[n]) n0 = n;
      if (n0 >= 0)
        for (size_t c = 0; c < cols.size(); ++c) ld[c] = cols[c].fs[n0];
      for (int n = 0; n < nf; ++n) {
        bool same = true;
        for (auto& c : cols) same = same && c.fs[n] == cols[0].fs[n];
        if (same) {
          sb[n] = cols[0].fs[n];
          continue;
        }
        if (ld[0] <= 0 || cols[0].fs[n] % ld[0]) return false;
        sa[n] = cols[0].fs[n] / ld[0];
        for (size_t c = 0; c < cols.size(); ++c)
          if (cols[c].fs[n] != ld[c] * sa[n]) return false;
      }
      for (int n = 0; n < nf; ++n)
        if (sa[n] >= ((int64_t)1 << 31) || sb[n] >= ((int64_t)1 << 31)) return false;
      return true;
    };
    auto plan_direct = [&](const G& g) -> bool {
      const int x = g.x;
      std::vector<int64_t> koff(g.k * g.n, 0);
      std::vector<double> kcoef(g.k * g.n, 0.0);
      for (int64_t sb : bsec[x]) {  // B_x[c][j] -> B offset and coefficient
        if (XB[sb].empty()) continue;
        if (XB[sb].size() != 1) return false;
        const int64_t src = XB[sb][0].first;
        group_weights(Bm, sb, nc, rw, cw);
        block_strides(B, src, st);
        std::vector<int> dims(Bm.rank);
        for (int n = 0; n < Bm.rank; ++n) dims[n] = Bm.dim(sb, n);
        each(dims, 0, Bm.rank, [&](const int* t) {
          int64_t r = MB.r0[sb], c = MB.c0[sb], off = B.offs[src];
          for (int n = 0; n < Bm.rank; ++n) {
            r += (int64_t)t[n] * rw[n];
            c += (int64_t)t[n] * cw[n];
            off += (int64_t)t[n] * st[permB[n]];
          }
          koff[r * g.n + c] = off;
          kcoef[r * g.n + c] = XB[sb][0].second;
        });
      }
      std::vector<DirectItem> f, ba, bb;
      for (auto& rk : arow[x]) {
        std::vector<Col> ac, cc;
        std::vector<int> fd(na, 1);
        for (int64_t s : rk.second) {  // A columns: contracted positions of each block
          if (XA[s].empty()) continue;
          if (XA[s].size() != 1 || std::fabs(XA[s][0].second) != 1.0) return false;
          const int64_t src = XA[s][0].first;
          const double sgn = XA[s][0].second;
          group_weights(Am, s, na, rw, cw);
          block_strides(A, src, st);
          std::vector<int> dims(Am.rank);
          std::vector<int64_t> fs(na);
          for (int n = 0; n < Am.rank; ++n) dims[n] = Am.dim(s, n);
          for (int n = 0; n < na; ++n) {
            fd[n] = dims[n];
            fs[n] = st[permA[n]];
          }
          each(dims, na, Am.rank, [&](const int* t) {
            int64_t c = MA.c0[s], off = A.offs[src];
            for (int n = na; n < Am.rank; ++n) {
              c += (int64_t)t[n] * cw[n];
              off += (int64_t)t[n] * st[permA[n]];
            }
            ac.push_back(Col{c, off, fs, sgn});
          });
        }
        auto ci = crow[x].find(rk.first);
        if (ci != crow[x].end())
          for (int64_t sn : ci->second) {  // C columns: B-free positions of each block
            group_weights(Cn, sn, na, rw, cw);
            block_strides(C, sn, st);
            std::vector<int> dims(Cn.rank);
            std::vector<int64_t> fs(na);
            for (int n = 0; n < Cn.rank; ++n) dims[n] = Cn.dim(sn, n);
            for (int n = 0; n < na; ++n) {
              if (dims[n] != fd[n]) return false;
              fs[n] = st[n];
            }
            const int64_t c0 = MB.coloff.at({x, col_key(Cn, sn, na)});
            each(dims, na, Cn.rank, [&](const int* t) {
              int64_t c = c0, off = C.offs[sn];
              for (int n = na; n < Cn.rank; ++n) {
                c += (int64_t)t[n] * cw[n];
                off += (int64_t)t[n] * st[n];
              }
              cc.push_back(Col{c, off, fs});
            });
          }
        if (ac.empty() && cc.empty()) continue;
        if (ac.empty() || cc.empty()) return false;  // a side without columns: leave x to the general path
        if ((int)ac.size() > kMaxDirect || (int)cc.size() > kMaxDirect) return false;
        std::vector<int64_t> ald, asa, asb, cld, csa, csb;
        if (!fit(ac, na, ald, asa, asb) || !fit(cc, na, cld, csa, csb)) return false;
        Box box;
        for (int n = 0; n < na; ++n) box.push(fd[n], (int)asa[n], (int)asb[n], (int)csa[n], (int)csb[n]);
        box = simplify(box);
        // peel leading dims beyond kDirectDims into offset shifts
        std::vector<std::pair<std::vector<int64_t>, std::vector<int64_t>>> origins;
        {
          std::vector<int64_t> so, dof;
          for (auto& c : ac) so.push_back(c.off);
          for (auto& c : cc) dof.push_back(c.off);
          origins.push_back({so, dof});
        }
        while (box.ndim > kDirectDims) {
          std::vector<std::pair<std::vector<int64_t>, std::vector<int64_t>>> next;
          for (auto& o : origins)
            for (int i = 0; i < box.dims[0]; ++i) {
              auto so = o.first, dof = o.second;
              for (size_t c = 0; c < so.size(); ++c) so[c] += (int64_t)i * (ald[c] * box.sa[0] + box.sb[0]);
              for (size_t c = 0; c < dof.size(); ++c) dof[c] += (int64_t)i * (cld[c] * box.da[0] + box.db[0]);
              next.push_back({so, dof});
            }
          origins.swap(next);
          Box b2;
          for (int d = 1; d < box.ndim; ++d) b2.push(box.dims[d], box.sa[d], box.sb[d], box.da[d], box.db[d]);
          box = b2;
        }
        int64_t total = 1, span = 0;
        for (int d = 0; d < box.ndim; ++d) total *= box.dims[d];
        for (int d = 0; d < box.ndim; ++d)
          span = std::max({span, (int64_t)(box.dims[d] - 1) * box.sa[d], (int64_t)(box.dims[d] - 1) * box.sb[d],
                           (int64_t)(box.dims[d] - 1) * box.da[d], (int64_t)(box.dims[d] - 1) * box.db[d]});
        if (total >= ((int64_t)1 << 31) || span * kDirectDims >= ((int64_t)1 << 31)) return false;
        const int ns = (int)ac.size(), nd = (int)cc.size();
        for (auto& o : origins) {
          // inline column records: A side (source of the forward and of dB,
          // destination of dA), C side (destination of the forward, source
          // of dA, second source of dB); coefficient (c, j) = B_x[c][j]
          DirectCol acol[kMaxDirect] = {}, ccol[kMaxDirect] = {};
          for (int c = 0; c < ns; ++c) {
            acol[c].off = o.first[c];
            for (int d = 0; d < box.ndim; ++d) acol[c].str[d] = (int32_t)(ald[c] * box.sa[d] + box.sb[d]);
          }
          for (int j = 0; j < nd; ++j) {
            ccol[j].off = o.second[j];
            for (int d = 0; d < box.ndim; ++d) ccol[j].str[d] = (int32_t)(cld[j] * box.da[d] + box.db[d]);
          }
          auto item = [&](int op, bool a_src, int slots, int64_t st0, int64_t cnt) {
            DirectItem it{};
            it.op = op;
            it.ns = a_src ? ns : nd;
            it.nd = a_src ? nd : ns;
            it.ndim = box.ndim;
            it.start = (int)st0;
            it.count = (int)cnt;
            it.slots = slots;
            for (int d = 0; d < kDirectDims; ++d) {
              it.dims[d] = d < box.ndim ? box.dims[d] : 1;
              int8_t sh;
              div_magic(it.dims[d], it.mag[d], sh);
              it.shf |= (int)(uint8_t)sh << (8 * d);
            }
            for (int c = 0; c < kMaxDirect; ++c) {
              it.src[c] = a_src ? acol[c] : ccol[c];
              it.dst[c] = a_src ? ccol[c] : acol[c];
            }
            // coefficient (d, s): the item's d-th destination and s-th source
            for (int d = 0; d < it.nd; ++d)
              for (int s2 = 0; s2 < it.ns; ++s2) {
                const int c = a_src ? s2 : d, j = a_src ? d : s2;
                const int64_t e = ac[c].idx * g.n + cc[j].idx;
                it.koff[d * kMaxDirect + s2] = koff[e];
                // the A column's sign enters every product it is in: C, dA and dB
                it.kc[d * kMaxDirect + s2] = kcoef[e] * ac[c].sgn;
              }
            return it;
          };
          for (int64_t p0 = 0; p0 < total; p0 += tp.direct_chunk) {
            const int64_t cnt = std::min<int64_t>(tp.direct_chunk, total - p0);
            // C = A B: sources A (slot 0), coefficients B (slot 1), destination C
            f.push_back(item(kDirectApply, true, 0 | (1 << 2) | (DST_OUT << 4), p0, cnt));
            // dA = dC B^T: sources dC (slot 2), coefficients B, destination dA
            ba.push_back(item(kDirectApply, false, 2 | (1 << 2) | (DST_DA << 4), p0, cnt));
          }
          const int64_t oc = 2 * (int64_t)tp.direct_chunk;  // outer items: one set of atomics each
          for (int64_t p0 = 0; p0 < total; p0 += oc) {
            const int64_t cnt = std::min<int64_t>(oc, total - p0);
            // dB += A^T dC: sources A (slot 0) and dC (slot 2), sums into dB
            bb.push_back(item(kDirectOuter, true, 0 | (2 << 2) | (DST_DB << 4), p0, cnt));
          }
        }
      }
      dfw.insert(dfw.end(), f.begin(), f.end());
      dba.insert(dba.end(), ba.begin(), ba.end());
      dbb.insert(dbb.end(), bb.begin(), bb.end());
      return true;
    };
    bool all = true;  // every sector qualifies for the direct path
    for (auto& g : gs) all = all && g.k <= dmax && g.n <= dmax;
    const bool use = all || tp.direct_mixed;
    std::vector<G> keep;
    for (auto& g : gs) {
      if (use && g.k <= dmax && g.n <= dmax && plan_direct(g)) {
        dset.insert(g.x);
        P->flops_fwd += 2.0 * (double)g.m * (double)g.n * (double)g.k;
      } else {
        keep.push_back(g);
      }
    }
    gs.swap(keep);
    gofx.clear();
    for (size_t i = 0; i < gs.size(); ++i) gofx[gs[i].x] = (int)i;
  }
  P->fwd_direct = {0, (int)dfw.size()};
  P->bwd_direct_a = {(int)dfw.size(), (int)dba.size()};
  P->bwd_direct_b = {(int)(dfw.size() + dba.size()), (int)dbb.size()};
  P->ditems = dfw;
  P->ditems.insert(P->ditems.end(), dba.begin(), dba.end());
  P->ditems.insert(P->ditems.end(), dbb.begin(), dbb.end());
  int64_t ie = 0, le = 0, oe = 0;
  auto ld64 = [](int64_t cols) { return cdiv(cols, 64) * 64; };  // rows on 128-byte lines
  // split-BF16 buffer of rows x cols bf16 in the hi plane
  auto add_buf = [&](int64_t rows, int64_t cols) {
    const int64_t off = ie;
    ie += rows * ld64(cols);
    return off;
  };
  // tensor map of a buffer (rows x cols stored): K-major or MN-major view
  auto add_op = [&](int64_t off, int64_t rows, int64_t cols, int mn) {
    P->tc_ops.push_back(TcOperand{off, (int)rows, (int)cols, (int)ld64(cols), mn});
    return (int)P->tc_ops.size() - 1;
  };
  for (auto& g : gs) {
    const bool t0 = g.kind[0] == 0, t1 = g.kind[1] == 0, t2 = g.kind[2] == 0;
    if (t0 || t2) g.ta = add_buf(g.m, g.k);
    if (t0 || t1) g.tb = add_buf(g.k, g.n);
    if (t1 || t2) g.tdc = add_buf(g.m, g.n);
    if (t0) {
      g.fa = add_op(g.ta, g.m, g.k, 0);
      g.fb = add_op(g.tb, g.k, g.n, 1);
    } else {
      g.a = le, le += g.m * g.k;
      g.b = le, le += g.k * g.n;
    }
    // the rows and thin kernels read the forward's linear B (dA = dC B^T) and
    // the thin kernel its linear A (dB = A^T dC) transposed, in place of
    // gathered transposed copies
    const bool reuse_b = !t0 && (g.kind[1] == 3 || g.kind[1] == 4);
    const bool reuse_a = !t0 && g.kind[2] == 3;
    if (t1) {
      g.dAa = add_op(g.tdc, g.m, g.n, 0);
      g.dAb = add_op(g.tb, g.k, g.n, 0);
    } else if (!reuse_b) {
      g.bt = le, le += g.n * g.k;
    }
    if (t2) {
      g.dBa = add_op(g.ta, g.m, g.k, 1);
      g.dBb = add_op(g.tdc, g.m, g.n, 1);
    } else if (!reuse_a) {
      g.at = le, le += g.k * g.m;
    }
    if (!t1 || !t2) g.dcl = le, le += g.m * g.n;
    if ((t0 && (t1 || t2)) || reuse_a || reuse_b) P->bwd_reads_fwd_operands = true;
  }
  for (auto& g : gs) {
    g.c = oe, oe += g.m * g.n;
    g.da = oe, oe += g.m * g.k;
    g.db = oe, oe += g.k * g.n;
  }
  P->img_elems = cdiv(ie, 64) * 64;  // the lo plane starts 128-byte aligned
  P->lin_elems = le;
  P->outm_elems = oe;
  for (auto& g : gs) P->flops_fwd += 2.0 * (double)g.m * (double)g.n * (double)g.k;
  P->numel_a = A.numel();
  P->numel_b = B.numel();
  P->numel_c = C.numel();

  // ---- GEMM sectors and tiles: lists per (kind, gemm phase)
  std::vector<std::pair<int64_t, GemmTile>> lists[kGemmKinds][3];
  const int nsm = 152;
  // kind 0: aoff, boff are tcgen05 operand indices; otherwise linear offsets
  auto add_gemm = [&](int kind, int ph, int64_t m, int64_t n, int64_t k, int64_t aoff, int64_t lda, int64_t boff,
                      int64_t ldb, int64_t coff, int trans) -> bool {
    if (kind == 0) {
      const int amn = P->tc_ops[aoff].mn, bmn = P->tc_ops[boff].mn;
      P->secs_tc.push_back(
          TcSector{(int)m, (int)n, (int)k, (int)cdiv(k, 64), (int)aoff, (int)boff, amn, bmn, coff, (int)n, 1.0f});
      const int sec = (int)P->secs_tc.size() - 1;
      // grouped order: tc_group row tiles at a time, all column tiles of the
      // group before the next (a wave of consecutive tiles shares panels)
      const int64_t MT = cdiv(m, 128), NT = cdiv(n, 128), G = tp.tc_group > 0 ? tp.tc_group : 1;
      for (int64_t g0 = 0; g0 < MT; g0 += G)
        for (int64_t nt = 0; nt < NT; ++nt)
          for (int64_t mt = g0; mt < std::min(MT, g0 + G); ++mt)
            lists[0][ph].push_back({k, GemmTile{sec, (int)mt, (int)nt, 0, (int)k, 0}});
      return false;
    }
    P->secs_simt.push_back(
        GemmSectorSimt{(int)m, (int)n, (int)k, (int)lda, (int)ldb, (int)n, aoff, boff, coff, 1.0, trans, 0});
    const int sec = (int)P->secs_simt.size() - 1;
    if (kind == 4) {  // rows: per-warp tiles of whole rows, whole (short) reduction
      const int64_t tr = (int64_t)tp.rows_spans * rows_span((int)k);
      for (int64_t r0 = 0; r0 < m; r0 += tr) {
        const int64_t r1 = std::min(m, r0 + tr);
        lists[4][ph].push_back({(r1 - r0) * (k + n), GemmTile{sec, 0, 0, (int)r0, (int)r1, 0}});
      }
      return false;
    }
    if (kind == 3) {  // thin: one CTA per 4096-long slice of the reduction
      const int64_t kc = tp.thin_slice, nsplit = cdiv(k, kc);
      for (int64_t sp = 0; sp < nsplit; ++sp) {
        const int64_t k0 = sp * kc, k1 = std::min(k, k0 + kc);
        lists[3][ph].push_back({k1 - k0, GemmTile{sec, 0, 0, (int)k0, (int)k1, nsplit > 1 ? 1 : 0}});
      }
      return nsplit > 1;
    }
    const int64_t TM = kind == 1 ? 64 : 256, TN = kind == 1 ? 64 : 16;
    const int64_t ntl = cdiv(m, TM) * cdiv(n, TN);
    int64_t nsplit = 1;
    const int64_t want = (int64_t)tp.splitk_ctas * nsm;  // CTAs a launch should reach by splitting k
    if (k >= 256 && ntl < want) nsplit = std::min<int64_t>(cdiv(k, 128), cdiv(want, ntl));
    const int64_t kc = cdiv(cdiv(k, nsplit), 32) * 32;
    nsplit = cdiv(k, kc);
    for (int64_t mt = 0; mt < cdiv(m, TM); ++mt)
      for (int64_t nt = 0; nt < cdiv(n, TN); ++nt)
        for (int64_t s = 0; s < nsplit; ++s) {
          const int64_t k0 = s * kc, k1 = std::min(k, k0 + kc);
          lists[kind][ph].push_back({k1 - k0, GemmTile{sec, (int)mt, (int)nt, (int)k0, (int)k1, nsplit > 1 ? 1 : 0}});
        }
    return nsplit > 1;
  };
  for (auto& g : gs) {
    const bool t0 = g.kind[0] == 0, t1 = g.kind[1] == 0, t2 = g.kind[2] == 0;
    g.split[0] = add_gemm(g.kind[0], 0, g.m, g.n, g.k, t0 ? g.fa : g.a, g.k, t0 ? g.fb : g.b, g.n, g.c, 0);
    if (t1 || g.bt >= 0)
      g.split[1] = add_gemm(g.kind[1], 1, g.m, g.k, g.n, t1 ? g.dAa : g.dcl, g.n, t1 ? g.dAb : g.bt, g.k, g.da, 0);
    else  // B^T read from the forward's B (k x n)
      g.split[1] = add_gemm(g.kind[1], 1, g.m, g.k, g.n, g.dcl, g.n, g.b, g.n, g.da, kTransB);
    if (t2 || g.at >= 0)
      g.split[2] = add_gemm(g.kind[2], 2, g.k, g.n, g.m, t2 ? g.dBa : g.at, g.m, t2 ? g.dBb : g.dcl, g.n, g.db, 0);
    else  // A^T read from the forward's A (m x k)
      g.split[2] = add_gemm(g.kind[2], 2, g.k, g.n, g.m, g.a, g.k, g.dcl, g.n, g.db, kTransA);
  }
  for (int kind = 0; kind < kGemmKinds; ++kind)
    for (int ph = 0; ph < 3; ++ph) {
      auto& v = lists[kind][ph];
      if (kind != 0 || tp.tc_order == 0)  // longest reductions first
        std::stable_sort(v.begin(), v.end(), [](auto& a, auto& b) { return a.first > b.first; });
      P->gemm_range[kind][ph] = Range{(int)P->tiles.size(), (int)v.size()};
      for (auto& t : v) {
        P->tiles.push_back(t.second);
        P->tile_kind.push_back(kind);
      }
    }

  std::vector<int> pinvA(A.rank), pinvB(B.rank);
  for (int n = 0; n < A.rank; ++n) pinvA[permA[n]] = n;
  for (int n = 0; n < B.rank; ++n) pinvB[permB[n]] = n;

  // box of a source block of S gathered into the matrix form of Sm (S leg l -> Sm leg pinv[l]);
  // swap_rc exchanges the roles of row and column weights (transposed operands)
  auto gather_box = [&](const Tensor& S, const std::vector<int>& pinv, const Tensor& Sm, int64_t sm, int64_t ssrc,
                        int nrows, bool swap_rc) {
    group_weights(Sm, sm, nrows, rw, cw);
    block_strides(S, ssrc, st);
    Box b;
    for (int l = 0; l < S.rank; ++l) {
      int n = pinv[l];
      b.push(S.dim(ssrc, l), st[l], 0, swap_rc ? cw[n] : rw[n], swap_rc ? rw[n] : cw[n]);
    }
    return b;
  };
  auto terms_of = [&](const TermList& tl, const Tensor& S) {
    std::vector<Term> t;
    for (auto& pc : tl) t.push_back({S.offs[pc.first], 1, pc.second});
    return t;
  };
  // operand block written into a linear matrix (row stride ld) at (row0, col0)
  auto put = [&](const Box& b, int src, int64_t off, int64_t row0, int64_t col0, int64_t ld,
                 const std::vector<Term>& t) { emit(*P, b, off + row0 * ld + col0, (int)ld, src, DST_OPS, t); };
  // operand block written into a split-BF16 buffer (rows of `cols`) at (row0, col0)
  auto put_tc = [&](const Box& b, int src, int64_t off, int64_t cols, int64_t row0, int64_t col0,
                    const std::vector<Term>& t) {
    emit(*P, b, off + row0 * ld64(cols) + col0, (int)ld64(cols), src, DST_SPLIT, t);
  };
  // zero-fill of an output matrix before a split-K GEMM adds into it
  auto zero_fill = [&](int64_t off, int64_t rows, int64_t cols) {
    Box b;
    b.push((int)rows, 0, 0, 1, 0);
    b.push((int)cols, 0, 0, 0, 1);
    emit(*P, b, off, (int)cols, 3, DST_OUTM, {});
  };

  using OffLd = std::pair<int64_t, int64_t>;
  auto fuse_recoupling = [&](int64_t ndst, const std::vector<TermList>& X, int src_slot,
                             const std::function<bool(int64_t, OffLd&, int&)>& dst_of,
                             const std::function<OffLd(int64_t)>& src_of,
                             const std::function<Box(int64_t, int64_t)>& box_of, std::vector<char>& done) {
    done.assign(ndst, 0);
    if (su2) fuse_recoupling_items(*P, ndst, X, src_slot, dst_of, src_of, box_of, done);
  };

  // ---- forward gather: A -> A operand, B -> B operand (+ zero fills)
  int begin = (int)P->items.size();
  std::vector<char> doneA;
  fuse_recoupling(
      Am.nsec(), XA, 0,
      [&](int64_t s, OffLd& o, int& slot) {
        auto gi = gofx.find(MA.xs[MA.sx[s]]);
        if (gi == gofx.end()) return false;
        const G& g = gs[gi->second];
        if (g.kind[0] == 0) {
          o = {g.ta + MA.r0[s] * ld64(g.k) + MA.c0[s], ld64(g.k)};
          slot = DST_SPLIT;
        } else {
          o = {g.a + MA.r0[s] * g.k + MA.c0[s], g.k};
          slot = DST_OPS;
        }
        return true;
      },
      [&](int64_t sa) { return OffLd{A.offs[sa], 1}; },
      [&](int64_t s, int64_t sa) { return gather_box(A, pinvA, Am, s, sa, na, false); }, doneA);
  for (int64_t s = 0; s < Am.nsec(); ++s) {
    auto gi = gofx.find(MA.xs[MA.sx[s]]);
    if (gi == gofx.end() || XA[s].empty() || doneA[s]) continue;
    const G& g = gs[gi->second];
    Box b = gather_box(A, pinvA, Am, s, XA[s][0].first, na, false);
    if (g.kind[0] == 0)
      put_tc(b, 0, g.ta, g.k, MA.r0[s], MA.c0[s], terms_of(XA[s], A));
    else
      put(b, 0, g.a, MA.r0[s], MA.c0[s], g.k, terms_of(XA[s], A));
  }
  for (int64_t s = 0; s < Bm.nsec(); ++s) {
    auto gi = gofx.find(MB.xs[MB.sx[s]]);
    if (gi == gofx.end() || XB[s].empty()) continue;
    const G& g = gs[gi->second];
    Box b = gather_box(B, pinvB, Bm, s, XB[s][0].first, nc, false);  // B (k x n)
    if (g.kind[0] == 0)
      put_tc(b, 1, g.tb, g.n, MB.r0[s], MB.c0[s], terms_of(XB[s], B));
    else
      put(b, 1, g.b, MB.r0[s], MB.c0[s], g.n, terms_of(XB[s], B));
  }
  for (auto& g : gs)
    if (g.split[0]) zero_fill(g.c, g.m, g.n);
  split_few_recouple_items(*P, begin);
  P->fwd_gather = {begin, (int)P->items.size() - begin};

  // ---- forward scatter: C_x -> C blocks (SU(2): Gamma to the requested tree)
  auto cn_term = [&](int64_t sn, double coef, std::vector<Term>& t) {
    auto gi = gofx.find(MC.xs[MC.sx[sn]]);
    if (gi == gofx.end()) return;
    const G& g = gs[gi->second];
    int x = MC.xs[MC.sx[sn]];
    int64_t r0 = MA.rowoff.at({x, row_key(Cn, sn, na)});
    int64_t c0 = MB.coloff.at({x, col_key(Cn, sn, na)});
    t.push_back({g.c + r0 * g.n + c0, g.n, coef});
  };
  begin = (int)P->items.size();
  for (int64_t s = 0; s < C.nsec(); ++s) {
    if (natural && dset.count(MC.xs[MC.sx[s]])) continue;  // written by the direct kernel
    std::vector<Term> t;
    if (natural) {
      cn_term(s, 1.0, t);
    } else {
      for (auto& pc : XC[s]) cn_term(pc.first, pc.second, t);
    }
    group_weights(C, s, na, rw, cw);
    block_strides(C, s, st);
    Box b;
    for (int l = 0; l < C.rank; ++l) b.push(C.dim(s, l), rw[l], cw[l], st[l], 0);
    emit(*P, b, C.offs[s], 1, 3, DST_OUT, t);
  }
  P->fwd_scatter = {begin, (int)P->items.size() - begin};

  // ---- backward gathers: [dA only: B or B^T][shared: dC][dB only: A or A^T]
  std::vector<int> idC(C.rank);
  for (int i = 0; i < C.rank; ++i) idC[i] = i;
  auto dc_terms = [&](int64_t sn) {
    std::vector<Term> t;
    if (natural) {
      t.push_back({C.offs[sn], 1, 1.0});
    } else {
      for (auto& pc : XCt[sn]) t.push_back({C.offs[pc.first], 1, pc.second});
    }
    return t;
  };
  auto for_dc = [&](const std::function<void(const G&, int64_t, int64_t, int64_t)>& fn) {
    for (int64_t sn = 0; sn < Cn.nsec(); ++sn) {
      auto gi = gofx.find(MC.xs[MC.sx[sn]]);
      if (gi == gofx.end()) continue;
      const G& g = gs[gi->second];
      int x = MC.xs[MC.sx[sn]];
      fn(g, sn, MA.rowoff.at({x, row_key(Cn, sn, na)}), MB.coloff.at({x, col_key(Cn, sn, na)}));
    }
  };
  const int b0 = (int)P->items.size();
  for (int64_t s = 0; s < Bm.nsec(); ++s) {
    auto gi = gofx.find(MB.xs[MB.sx[s]]);
    if (gi == gofx.end() || XB[s].empty()) continue;
    const G& g = gs[gi->second];
    if (g.kind[1] == 0) {  // B (k x n) for the tensor cores, unless the forward wrote it
      if (g.kind[0] == 0) continue;
      Box b = gather_box(B, pinvB, Bm, s, XB[s][0].first, nc, false);
      put_tc(b, 1, g.tb, g.n, MB.r0[s], MB.c0[s], terms_of(XB[s], B));
    } else if (g.bt >= 0) {  // B^T (n x k), unless the GEMM reads the forward's B
      Box b = gather_box(B, pinvB, Bm, s, XB[s][0].first, nc, true);
      put(b, 1, g.bt, MB.c0[s], MB.r0[s], g.k, terms_of(XB[s], B));
    }
  }
  for (auto& g : gs)
    if (g.split[1]) zero_fill(g.da, g.m, g.k);
  const int b1 = (int)P->items.size();
  for_dc([&](const G& g, int64_t sn, int64_t r0, int64_t c0) {  // dC (m x n), both gradients
    auto t = dc_terms(sn);
    if (t.empty()) return;
    Box b = gather_box(Cn, idC, Cn, sn, sn, na, false);
    if (g.tdc >= 0) put_tc(b, 2, g.tdc, g.n, r0, c0, t);
    if (g.dcl >= 0) put(b, 2, g.dcl, r0, c0, g.n, t);
  });
  const int b2 = (int)P->items.size();
  for (int64_t s = 0; s < Am.nsec(); ++s) {
    auto gi = gofx.find(MA.xs[MA.sx[s]]);
    if (gi == gofx.end() || XA[s].empty()) continue;
    const G& g = gs[gi->second];
    if (g.kind[2] == 0) {  // A (m x k) for the tensor cores, unless the forward wrote it
      if (g.kind[0] == 0) continue;
      Box b = gather_box(A, pinvA, Am, s, XA[s][0].first, na, false);
      put_tc(b, 0, g.ta, g.k, MA.r0[s], MA.c0[s], terms_of(XA[s], A));
    } else if (g.at >= 0) {  // A^T (k x m), unless the GEMM reads the forward's A
      Box b = gather_box(A, pinvA, Am, s, XA[s][0].first, na, true);
      put(b, 0, g.at, MA.c0[s], MA.r0[s], g.m, terms_of(XA[s], A));
    }
  }
  for (auto& g : gs)
    if (g.split[2]) zero_fill(g.db, g.k, g.n);
  const int b3 = (int)P->items.size();
  P->bwd_gather_a = {b0, b2 - b0};
  P->bwd_gather_b = {b1, b3 - b1};

  // ---- backward scatters: dA_x -> dA blocks (Gamma^T), dB_x -> dB blocks
  begin = (int)P->items.size();
  std::vector<char> doneDA;
  fuse_recoupling(
      A.nsec(), XAt, 3,
      [&](int64_t s, OffLd& o, int& slot) {
        for (auto& pc : XAt[s])
          if (gofx.find(MA.xs[MA.sx[pc.first]]) == gofx.end()) return false;
        o = {A.offs[s], 1};
        slot = DST_DA;
        return true;
      },
      [&](int64_t sm) {
        const G& g = gs[gofx.at(MA.xs[MA.sx[sm]])];
        return OffLd{g.da + MA.r0[sm] * g.k + MA.c0[sm], g.k};
      },
      [&](int64_t s, int64_t sm) {
        group_weights(Am, sm, na, rw, cw);
        block_strides(A, s, st);
        Box b;
        for (int l = 0; l < A.rank; ++l) b.push(A.dim(s, l), rw[pinvA[l]], cw[pinvA[l]], st[l], 0);
        return b;
      },
      doneDA);
  for (int64_t s = 0; s < A.nsec(); ++s) {
    if (doneDA[s]) continue;
    bool direct = false;  // dA written by the direct kernel
    for (auto& pc : XAt[s]) direct = direct || dset.count(MA.xs[MA.sx[pc.first]]) > 0;
    if (direct) continue;
    std::vector<Term> t;
    int64_t sm0 = -1;
    for (auto& pc : XAt[s]) {
      int64_t sm = pc.first;
      auto gi = gofx.find(MA.xs[MA.sx[sm]]);
      if (gi == gofx.end()) continue;
      const G& g = gs[gi->second];
      t.push_back({g.da + MA.r0[sm] * g.k + MA.c0[sm], g.k, pc.second});
      if (sm0 < 0) sm0 = sm;
    }
    block_strides(A, s, st);
    Box b;
    if (sm0 >= 0) group_weights(Am, sm0, na, rw, cw);
    for (int l = 0; l < A.rank; ++l) {
      int n = pinvA[l];
      b.push(A.dim(s, l), sm0 >= 0 ? rw[n] : 0, sm0 >= 0 ? cw[n] : 0, st[l], 0);
    }
    emit(*P, b, A.offs[s], 1, 3, DST_DA, t);
  }
  split_few_recouple_items(*P, begin);
  P->bwd_scatter_a = {begin, (int)P->items.size() - begin};
  begin = (int)P->items.size();
  for (int64_t s = 0; s < B.nsec(); ++s) {
    std::vector<Term> t;
    int64_t sm0 = -1;
    for (auto& pc : XBt[s]) {
      int64_t sm = pc.first;
      auto gi = gofx.find(MB.xs[MB.sx[sm]]);
      if (gi == gofx.end()) continue;
      const G& g = gs[gi->second];
      t.push_back({g.db + MB.r0[sm] * g.n + MB.c0[sm], g.n, pc.second});
      if (sm0 < 0) sm0 = sm;
    }
    block_strides(B, s, st);
    Box b;
    if (sm0 >= 0) group_weights(Bm, sm0, nc, rw, cw);
    for (int l = 0; l < B.rank; ++l) {
      int n = pinvB[l];
      b.push(B.dim(s, l), sm0 >= 0 ? rw[n] : 0, sm0 >= 0 ? cw[n] : 0, st[l], 0);
    }
    emit(*P, b, B.offs[s], 1, 3, DST_DB, t);
  }
  P->bwd_scatter_b = {begin, (int)P->items.size() - begin};
  {
    const int es = f64 ? 8 : 4;
    P->set_item_bytes({0, (int)P->items.size()}, es, es);
  }
  {
    const int64_t src[4] = {A.numel(), B.numel(), C.numel(), P->outm_elems};
    const int64_t dst[DST_COUNT] = {C.numel(), A.numel(), B.numel(), P->lin_elems, P->outm_elems, P->img_elems};
    P->validate(src, dst);
  }
  validate_gemms(*P, f64);
  validate_direct(*P);
  P->upload(device);
  return P;
}

// One plan running many independent contractions: the host plans (device =
// false) of problems i = 0..n-1 merged with their offsets shifted into packed
// buffers (problem i's A at offA[i] of the packed A, likewise B and C) and into
// shared scratch.  Every phase stays one launch per kernel over all problems:
// items are concatenated phase by phase (the backward gathers keep their
// dA-only / shared dC / dB-only order) and the GEMM tiles of each kind and
// phase are concatenated and re-sorted by reduction length (longest first).
std::unique_ptr<Plan> merge_contract_plans(std::vector<std::unique_ptr<Plan>>& ps, const std::vector<int64_t>& offA,
                                           const std::vector<int64_t>& offB, const std::vector<int64_t>& offC,
                                           bool device) {
  const int n = (int)ps.size();
  if (n < 1) fail(SYM_ERR_ARG, "empty batch");
  auto M = std::make_unique<Plan>();
  M->kind = Plan::CONTRACT;
  M->precision = ps[0]->precision;
  const bool f64 = M->precision == SYM_PREC_FP64;
  M->tc_order = ps[0]->tc_order;
  std::vector<int64_t> lin0(n), outm0(n), img0(n);
  std::vector<int> ops0(n), simt0(n), tc0(n);
  for (int i = 0; i < n; ++i) {
    const Plan& p = *ps[i];
    if (p.kind != Plan::CONTRACT || p.precision != M->precision) fail(SYM_ERR_ARG, "batch plans must match");
    lin0[i] = M->lin_elems;
    M->lin_elems += p.lin_elems;
    outm0[i] = M->outm_elems;
    M->outm_elems += p.outm_elems;
    img0[i] = M->img_elems;
    M->img_elems += cdiv(p.img_elems, 64) * 64;
    ops0[i] = (int)M->tc_ops.size();
    for (TcOperand o : p.tc_ops) {
      o.off += img0[i];
      M->tc_ops.push_back(o);
    }
    simt0[i] = (int)M->secs_simt.size();
    for (GemmSectorSimt g : p.secs_simt) {
      g.a_off += lin0[i];
      g.b_off += lin0[i];
      g.c_off += outm0[i];
      M->secs_simt.push_back(g);
    }
    tc0[i] = (int)M->secs_tc.size();
    for (TcSector g : p.secs_tc) {
      g.amap += ops0[i];
      g.bmap += ops0[i];
      g.c_off += outm0[i];
      M->secs_tc.push_back(g);
    }
    M->flops_fwd += p.flops_fwd;
    M->numel_a = offA[i] + p.numel_a;
    M->numel_b = offB[i] + p.numel_b;
    M->numel_c = offC[i] + p.numel_c;
    M->bwd_reads_fwd_operands |= p.bwd_reads_fwd_operands;
  }
  // items, with their term blocks copied once per problem
  std::vector<std::vector<int>> remap(n);
  for (int i = 0; i < n; ++i) remap[i].assign(ps[i]->terms.size(), -1);
  auto copy_range = [&](int i, int first, int count) {
    const Plan& p = *ps[i];
    const int64_t src_shift[4] = {offA[i], offB[i], offC[i], outm0[i]};
    const int64_t dst_shift[DST_COUNT] = {offC[i], offA[i], offB[i], lin0[i], outm0[i], img0[i]};
    for (int k = first; k < first + count; ++k) {
      BoxItem it = p.items[k];
      const int ss = it.sel & 3, ds = (it.sel >> 4) & 7;
      const bool rec = (it.sel & kSelRecouple) != 0;
      const int nt = rec ? it.nterm + it.p0 + it.nterm * it.p0 : it.nterm;
      if (nt > 0) {
        if (remap[i][it.term0] < 0) {
          remap[i][it.term0] = (int)M->terms.size();
          for (int q = 0; q < nt; ++q) {
            Term t = p.terms[it.term0 + q];
            if (!rec || q < it.nterm)
              t.off += src_shift[ss];
            else if (q < it.nterm + it.p0)
              t.off += dst_shift[ds];
            M->terms.push_back(t);
          }
        }
        it.term0 = remap[i][it.term0];
      } else {
        it.term0 = (int)M->terms.size();
      }
      if (!rec) {
        if (it.nterm > 0) it.t0_off += src_shift[ss];
        it.dst_off += dst_shift[ds];
      }
      M->items.push_back(it);
    }
  };
  auto concat = [&](const std::function<Range(const Plan&)>& sub) {
    const int first = (int)M->items.size();
    for (int i = 0; i < n; ++i) {
      const Range r = sub(*ps[i]);
      copy_range(i, r.first, r.count);
    }
    return Range{first, (int)M->items.size() - first};
  };
  M->fwd_gather = concat([](const Plan& p) { return p.fwd_gather; });
  M->fwd_scatter = concat([](const Plan& p) { return p.fwd_scatter; });
  // backward gathers: [a-only) [shared) [b-only)
  auto a_only = [](const Plan& p) { return Range{p.bwd_gather_a.first, p.bwd_gather_b.first - p.bwd_gather_a.first}; };
  auto shared = [](const Plan& p) {
    return Range{p.bwd_gather_b.first, p.bwd_gather_a.first + p.bwd_gather_a.count - p.bwd_gather_b.first};
  };
  auto b_only = [](const Plan& p) {
    const int e = p.bwd_gather_a.first + p.bwd_gather_a.count;
    return Range{e, p.bwd_gather_b.first + p.bwd_gather_b.count - e};
  };
  for (auto& pp : ps)
    if (a_only(*pp).count < 0 || shared(*pp).count < 0 || b_only(*pp).count < 0)
      fail(SYM_ERR_ARG, "internal: backward gather ranges out of order");
  const Range ra = concat(a_only), rs = concat(shared), rb = concat(b_only);
  M->bwd_gather_a = {ra.first, ra.count + rs.count};
  M->bwd_gather_b = {rs.first, rs.count + rb.count};
  M->bwd_scatter_a = concat([](const Plan& p) { return p.bwd_scatter_a; });
  M->bwd_scatter_b = concat([](const Plan& p) { return p.bwd_scatter_b; });
  // direct items: column and coefficient offsets shifted into the packed tensors
  {
    // tensor of a source slot (0 A, 1 B, 2 dC) and of a destination slot
    auto src_space = [](int slot) { return slot == 0 ? 0 : slot == 1 ? 1 : 2; };
    auto dst_space = [](int slot) { return slot == DST_OUT ? 2 : slot == DST_DA ? 0 : 1; };
    Range* dst[3] = {&M->fwd_direct, &M->bwd_direct_a, &M->bwd_direct_b};
    for (int r = 0; r < 3; ++r) {
      const int first = (int)M->ditems.size();
      for (int i = 0; i < n; ++i) {
        const Plan& p = *ps[i];
        const int64_t shift[3] = {offA[i], offB[i], offC[i]};
        const Range src = r == 0 ? p.fwd_direct : r == 1 ? p.bwd_direct_a : p.bwd_direct_b;
        for (int k = src.first; k < src.first + src.count; ++k) {
          DirectItem it = p.ditems[k];
          const int s1 = it.slots & 3, s2 = (it.slots >> 2) & 3, ds = (it.slots >> 4) & 7;
          const int64_t sh_src = shift[src_space(s1)];
          const int64_t sh_dst = shift[it.op == kDirectApply ? dst_space(ds) : src_space(s2)];
          const int64_t sh_k = shift[1];  // coefficients (apply) and outputs (outer) live in B / dB
          for (int c = 0; c < it.ns; ++c) it.src[c].off += sh_src;
          for (int c = 0; c < it.nd; ++c) it.dst[c].off += sh_dst;
          for (int e = 0; e < kMaxDirect * kMaxDirect; ++e)
            if (it.kc[e] != 0.0) it.koff[e] += sh_k;
          M->ditems.push_back(it);
        }
      }
      *dst[r] = Range{first, (int)M->ditems.size() - first};
    }
  }
  // GEMM tiles per (kind, phase), longest reductions first across problems
  for (int kind = 0; kind < kGemmKinds; ++kind)
    for (int ph = 0; ph < 3; ++ph) {
      std::vector<GemmTile> v;
      for (int i = 0; i < n; ++i) {
        const Range r = ps[i]->gemm_range[kind][ph];
        for (int t = r.first; t < r.first + r.count; ++t) {
          GemmTile g = ps[i]->tiles[t];
          g.sector += kind == 0 ? tc0[i] : simt0[i];
          v.push_back(g);
        }
      }
      if (kind != 0 || M->tc_order == 0)
        std::stable_sort(v.begin(), v.end(), [](const GemmTile& a, const GemmTile& b) { return a.k1 - a.k0 > b.k1 - b.k0; });
      M->gemm_range[kind][ph] = Range{(int)M->tiles.size(), (int)v.size()};
      for (auto& g : v) {
        M->tiles.push_back(g);
        M->tile_kind.push_back(kind);
      }
    }
  {
    const int es = f64 ? 8 : 4;
    M->set_item_bytes({0, (int)M->items.size()}, es, es);
    const int64_t src[4] = {M->numel_a, M->numel_b, M->numel_c, M->outm_elems};
    const int64_t dst[DST_COUNT] = {M->numel_c, M->numel_a, M->numel_b, M->lin_elems, M->outm_elems, M->img_elems};
    M->validate(src, dst);
  }
  validate_gemms(*M, f64);
  validate_direct(*M);
  M->upload(device);
  return M;
}

// ------------------------------------------------------------------- execution --
namespace {

int cuda_code(int e, const char* what) {
  if (e == 0) return SYM_OK;
  fail(SYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString((cudaError_t)e));
}

struct ProfScope {
  Plan& p;
  int phase, kernel;
  double bytes, flops;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s;
  ProfScope(Plan& p_, int ph, int kern, void* stream, double by, double fl)
      : p(p_), phase(ph), kernel(kern), bytes(by), flops(fl) {
    s = static_cast<cudaStream_t>(stream);
    if (!p.profiling) return;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    record(e0);
    p.prof[ph].launches++;
    p.prof[ph].bytes += bytes;
    p.prof[ph].flops += flops;
  }
  // inside a stream capture the events become external record nodes of the
  // graph, so every replay re-records them
  void record(cudaEvent_t e) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    if (st == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s);
  }
  ~ProfScope() {
    if (!p.profiling) return;
    record(e1);
    p.prof[phase].events.push_back(LaunchRecord{e0, e1, kernel, bytes, flops});
  }
};

int run_box(Plan& p, Range r, const BoxPtrs& ptrs, void* stream, int phase) {
  if (r.count <= 0) return SYM_OK;
  p.last_launches++;
  const int flat = p.flat_prefix[r.first + r.count] - p.flat_prefix[r.first];
  const int rec = p.recouple_prefix[r.first + r.count] - p.recouple_prefix[r.first];
  const int mode = flat == r.count ? kBoxFlat : flat + rec == r.count ? kBoxRecouple : kBoxGeneral;
  ProfScope ps(p, phase, mode == kBoxFlat ? SYM_KERNEL_BOX_FLAT : SYM_KERNEL_BOX, stream,
               p.item_bytes_prefix[r.first + r.count] - p.item_bytes_prefix[r.first], 0.0);
  return cuda_code(launch_box(p.f64(), p.f64(), mode, p.d_items + r.first, r.count, p.d_terms, ptrs, stream),
                   "box kernel");
}

// one launch per item kind (`op`): the apply and the outer items have kernels of their own
int run_direct(Plan& p, int op, Range r, const BoxPtrs& ptrs, void* stream, int phase) {
  if (r.count <= 0) return SYM_OK;
  p.last_launches++;
  ProfScope ps(p, phase, SYM_KERNEL_DIRECT, stream,
               p.ditem_bytes_prefix[r.first + r.count] - p.ditem_bytes_prefix[r.first],
               p.ditem_flops_prefix[r.first + r.count] - p.ditem_flops_prefix[r.first]);
  return cuda_code(launch_direct(p.f64(), op, p.d_ditems + r.first, r.count, ptrs, stream),
                   "direct kernel");
}

int run_gemm_kind(Plan& p, int kind, Range r, void* stream, int phase) {
  if (r.count <= 0) return SYM_OK;
  p.last_launches++;
  if (kind != 0) phase = phase == PH_FWD_GEMM ? PH_FWD_GEMM_SIMT : PH_BWD_GEMM_SIMT;
  static const int kernel_of_kind[kGemmKinds] = {SYM_KERNEL_GEMM_TC, SYM_KERNEL_GEMM_TILE, SYM_KERNEL_GEMM_WIDE,
                                                 SYM_KERNEL_GEMM_THIN, SYM_KERNEL_GEMM_ROWS};
  ProfScope ps(p, phase, kernel_of_kind[kind], stream,
               p.tile_bytes_prefix[r.first + r.count] - p.tile_bytes_prefix[r.first],
               p.tile_flops_prefix[r.first + r.count] - p.tile_flops_prefix[r.first]);
  if (kind == 0)
    return cuda_code(launch_gemm_tc(p.d_secs_tc, p.d_tiles + r.first, r.count, p.d_maps,
                                    static_cast<float*>(p.outm), p.d_err, stream),
                     "tcgen05 gemm");
  const int shape = kind == 1 ? SIMT_64x64 : kind == 2 ? SIMT_256x16 : kind == 3 ? SIMT_THIN : SIMT_ROWS;
  return cuda_code(launch_gemm_simt(p.f64(), shape, p.d_secs_simt,
                                    p.d_tiles + r.first, r.count, p.lin, p.outm, stream),
                   "cuda-core gemm");
}

// GEMM phases [ph0, ph1] (contiguous within each kind).  The kinds with
// work run concurrently: the first on `stream`, the others on the plan's
// side streams, forked from and joined back into `stream` with events.
int run_gemm(Plan& p, int ph0, int ph1, void* stream, int phase) {
  int kinds[kGemmKinds];
  Range rs[kGemmKinds];
  int n = 0;
  for (int kind = 0; kind < kGemmKinds; ++kind) {
    Range r{p.gemm_range[kind][ph0].first, 0};
    for (int ph = ph0; ph <= ph1; ++ph) r.count += p.gemm_range[kind][ph].count;
    if (r.count > 0) {
      kinds[n] = kind;
      rs[n++] = r;
    }
  }
  // while profiling, the kinds run one after another: each launch's event
  // pair then brackets that kernel alone (as a serialised profiler sees it)
  if (n <= 1 || !p.concurrent || p.profiling) {
    for (int i = 0; i < n; ++i)
      if (int rc = run_gemm_kind(p, kinds[i], rs[i], stream, phase)) return rc;
    return SYM_OK;
  }
  cudaStream_t s0 = static_cast<cudaStream_t>(stream);
  auto check = [](cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  if (!p.ev_fork) {
    cudaEvent_t e;
    check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    p.ev_fork = e;
  }
  for (int i = 0; i < n - 1; ++i) {
    if (!p.side[i]) {
      cudaStream_t st;
      check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate");
      p.side[i] = st;
    }
    if (!p.ev_join[i]) {
      cudaEvent_t e;
      check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
      p.ev_join[i] = e;
    }
  }
  check(cudaEventRecord(static_cast<cudaEvent_t>(p.ev_fork), s0), "cudaEventRecord");
  for (int i = 0; i < n - 1; ++i)
    check(cudaStreamWaitEvent(static_cast<cudaStream_t>(p.side[i]), static_cast<cudaEvent_t>(p.ev_fork), 0),
          "cudaStreamWaitEvent");
  int rc = run_gemm_kind(p, kinds[0], rs[0], stream, phase);
  for (int i = 1; i < n; ++i) {
    const int r = run_gemm_kind(p, kinds[i], rs[i], p.side[i - 1], phase);
    if (!rc) rc = r;
  }
  // join every side stream, also after a failed launch
  for (int i = 0; i < n - 1; ++i) {
    cudaEventRecord(static_cast<cudaEvent_t>(p.ev_join[i]), static_cast<cudaStream_t>(p.side[i]));
    cudaStreamWaitEvent(s0, static_cast<cudaEvent_t>(p.ev_join[i]), 0);
  }
  return rc;
}

BoxPtrs gather_ptrs(Plan& p, const void* A, const void* B, const void* dC) {
  BoxPtrs g{};
  g.src[0] = A;
  g.src[1] = B;
  g.src[2] = dC;
  g.src[3] = p.outm;
  g.dst[DST_OPS] = p.lin;
  g.dst[DST_OUTM] = p.outm;
  g.dst[DST_SPLIT] = p.img;
  g.split_lo = p.img_elems;
  return g;
}

}  // namespace

std::unique_ptr<Plan> chain_transforms(std::vector<std::unique_ptr<Plan>> steps, int precision) {
  if (steps.empty()) fail(SYM_ERR_ARG, "internal: empty transform chain");
  auto P = std::make_unique<Plan>();
  P->kind = Plan::TRANSFORM;
  P->precision = precision;
  P->numel_a = steps.front()->numel_a;
  P->numel_c = steps.back()->numel_c;
  P->dry = steps.front()->dry;
  int64_t mid = 1;  // the largest intermediate
  for (size_t i = 0; i + 1 < steps.size(); ++i) mid = std::max(mid, steps[i]->numel_c);
  P->chain = std::move(steps);
  if (!P->dry) {
    const size_t es = precision == SYM_PREC_FP64 ? sizeof(double) : sizeof(float);
    P->chain_buf[0] = P->arena.alloc((size_t)mid * es, false);
    P->chain_buf[1] = P->arena.alloc((size_t)mid * es, false);
  }
  return P;
}

int exec_transform(Plan& p, const void* in, void* out, void* stream) {
  if (p.dry) fail(SYM_ERR_UNSUPPORTED, "plan was built with SYM_PLAN_DRYRUN=1 and cannot run");
  p.last_launches = 0;
  if (!p.chain.empty()) {  // each step's output feeds the next, through the scratch pair
    const void* src = in;
    for (size_t i = 0; i < p.chain.size(); ++i) {
      void* dst = i + 1 == p.chain.size() ? out : p.chain_buf[i & 1];
      if (int rc = exec_transform(*p.chain[i], src, dst, stream)) return rc;
      p.last_launches += p.chain[i]->last_launches;
      src = dst;
    }
    return SYM_OK;
  }
  BoxPtrs ptrs{};
  ptrs.src[0] = in;
  ptrs.dst[DST_OUT] = out;
  return run_box(p, p.xform, ptrs, stream, PH_XFORM);
}

int exec_contract(Plan& p, const void* A, const void* B, void* C, void* stream) {
  if (p.dry) fail(SYM_ERR_UNSUPPORTED, "plan was built with SYM_PLAN_DRYRUN=1 and cannot run");
  p.last_launches = 0;
  BoxPtrs g = gather_ptrs(p, A, B, nullptr);
  int rc = run_box(p, p.fwd_gather, g, stream, PH_FWD_GATHER);
  if (rc) return rc;
  rc = run_gemm(p, 0, 0, stream, PH_FWD_GEMM);
  if (rc) return rc;
  p.fwd_a = A;
  p.fwd_b = B;
  BoxPtrs s{};
  s.src[3] = p.outm;
  s.dst[DST_OUT] = C;
  rc = run_box(p, p.fwd_scatter, s, stream, PH_FWD_SCATTER);
  if (rc) return rc;
  BoxPtrs d{};
  d.src[0] = A;
  d.src[1] = B;
  d.dst[DST_OUT] = C;
  return run_direct(p, kDirectApply, p.fwd_direct, d, stream, PH_FWD_DIRECT);
}

int exec_contract_backward(Plan& p, const void* A, const void* B, const void* dC, void* dA, void* dB,
                           void* stream) {
  if (p.dry) fail(SYM_ERR_UNSUPPORTED, "plan was built with SYM_PLAN_DRYRUN=1 and cannot run");
  p.last_launches = 0;
  if (!dA && !dB) return SYM_OK;
  BoxPtrs g = gather_ptrs(p, A, B, dC);
  if (p.bwd_reads_fwd_operands && (p.fwd_a != A || p.fwd_b != B)) {
    // the operand buffers hold another forward's inputs: gather A and B again
    if (int rc = run_box(p, p.fwd_gather, g, stream, PH_BWD_GATHER)) return rc;
    p.fwd_a = A;
    p.fwd_b = B;
  }
  Range gr;
  if (dA && dB) {
    int first = std::min(p.bwd_gather_a.first, p.bwd_gather_b.first);
    int last = std::max(p.bwd_gather_a.first + p.bwd_gather_a.count, p.bwd_gather_b.first + p.bwd_gather_b.count);
    gr = {first, last - first};
  } else {
    gr = dA ? p.bwd_gather_a : p.bwd_gather_b;
  }
  int rc = run_box(p, gr, g, stream, PH_BWD_GATHER);
  if (rc) return rc;
  rc = run_gemm(p, dA ? 1 : 2, dB ? 2 : 1, stream, PH_BWD_GEMM);
  if (rc) return rc;
  BoxPtrs s{};
  s.src[3] = p.outm;
  s.dst[DST_DA] = dA;
  s.dst[DST_DB] = dB;
  Range sr;
  if (dA && dB)
    sr = {p.bwd_scatter_a.first, p.bwd_scatter_a.count + p.bwd_scatter_b.count};
  else
    sr = dA ? p.bwd_scatter_a : p.bwd_scatter_b;
  rc = run_box(p, sr, s, stream, PH_BWD_SCATTER);
  if (rc) return rc;
  // after the scatter, which zero-filled the dB blocks the direct sums add into
  BoxPtrs d{};
  d.src[0] = A;
  d.src[1] = B;
  d.src[2] = dC;
  d.dst[DST_DA] = dA;
  d.dst[DST_DB] = dB;
  if (dA)
    if (int r = run_direct(p, kDirectApply, p.bwd_direct_a, d, stream, PH_BWD_DIRECT)) return r;
  return dB ? run_direct(p, kDirectOuter, p.bwd_direct_b, d, stream, PH_BWD_DIRECT) : SYM_OK;
}

}  // namespace sym
