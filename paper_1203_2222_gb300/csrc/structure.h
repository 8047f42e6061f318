// Host-side structure of symmetric tensors: legs, fusion trees, sector tables.
//
// Integer-exact bookkeeping only (no floating point).  The conventions are
// the ones stated in include/symtensor.h:
//   U(1)  sector = one charge position per leg, sum_out q - sum_in q == Q.
//   SU(2) sector = one spin position per leg + one spin per non-root node of
//         the fusion tree (Ch. 6, tree decompositions), every node obeying
//         the fusion rule (Ch. 5, Eq. fusionrules), root spin 0.
//   Sectors in lexicographic order (leg positions, leg 0 slowest; then node
//   spins in node order); blocks row-major and concatenated in that order.
#pragma once

#include <array>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/symtensor.h"

namespace sym {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void fail(int code, const std::string& msg);

// Groups whose tensors are tree decompositions (SU(2), and SU(2) x U(1)
// whose label 64 q + 2j carries a charge next to the spin).
inline bool su2_like(int group) { return group == SYM_SU2 || group == SYM_SU2U1; }
inline int spin_of(int group, int label) { return group == SYM_SU2U1 ? ((label % 64) + 64) % 64 : label; }
inline int charge_of(int group, int label) { return group == SYM_SU2U1 ? (label - spin_of(group, label)) / 64 : 0; }
inline int su2u1_label(int charge, int spin2) { return 64 * charge + spin2; }

struct Leg {
  std::vector<int> labels;  // U(1) charges or SU(2) doubled spins, increasing
  std::vector<int> degens;  // degeneracy of every label
  int dir = 1;              // +1 out, -1 in
  bool same_content(const Leg& o) const {
    return labels == o.labels && degens == o.degens;
  }
  int64_t degen_total() const {
    int64_t s = 0;
    for (int d : degens) s += d;
    return s;
  }
};

// Planar binary fusion tree over k legs: nodes[n] = {left id, right id};
// ids 0..k-1 are legs, node n has id k+n, the last node is the root.
struct Tree {
  int k = 0;
  std::vector<std::array<int, 2>> nodes;
  static Tree comb(int k);
  // comb over legs [0, na) and comb over [na, na+nb) joined at the root
  static Tree comb_pair(int na, int nb);
  void validate() const;  // throws sym::Error(SYM_ERR_ARG)
  bool operator==(const Tree& o) const { return k == o.k && nodes == o.nodes; }
};

struct VecHash {
  size_t operator()(const std::vector<int>& v) const {
    uint64_t h = 1469598103934665603ull;
    for (int x : v) {
      h ^= (uint64_t)(uint32_t)x;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

struct Tensor {
  int group = 0;  // SYM_U1, SYM_SU2, SYM_Z2F or SYM_SU2U1
  int rank = 0;
  std::vector<Leg> legs;
  int total = 0;  // U(1) total charge (SYM_SU2U1: the charge part)
  Tree tree;      // SU(2) and SU(2) x U(1)
  int nin = 0;    // SU(2) non-root node labels per sector (rank-2 for rank>=2)
  std::vector<int> pos;        // nsec * rank label positions
  std::vector<int> inner;      // nsec * nin node spins
  std::vector<int64_t> offs;   // nsec + 1
  std::unordered_map<std::vector<int>, int64_t, VecHash> index;

  int64_t nsec() const { return (int64_t)offs.size() - 1; }
  int64_t numel() const { return offs.back(); }
  int64_t block_size(int64_t s) const { return offs[s + 1] - offs[s]; }
  int p(int64_t s, int l) const { return pos[(size_t)s * rank + l]; }
  int label(int64_t s, int l) const { return legs[l].labels[p(s, l)]; }
  int dim(int64_t s, int l) const { return legs[l].degens[p(s, l)]; }
  const int* inner_of(int64_t s) const { return inner.data() + (size_t)s * nin; }
  // sector id of (positions, node spins), -1 if absent
  int64_t find(const std::vector<int>& key) const {
    auto it = index.find(key);
    return it == index.end() ? -1 : it->second;
  }
  std::vector<int> key(int64_t s) const {
    std::vector<int> k(pos.begin() + (size_t)s * rank, pos.begin() + (size_t)(s + 1) * rank);
    k.insert(k.end(), inner.begin() + (size_t)s * nin, inner.begin() + (size_t)(s + 1) * nin);
    return k;
  }
};

// Build the sector table.  Throws sym::Error on malformed input.
Tensor make_tensor(int group, const std::vector<Leg>& legs, int total, const Tree& tree);

// Enumerate the node-spin labelings (non-root nodes, node order, each spin
// ascending) of `tree` for fixed leg spins.  Root spin is 0.
std::vector<std::vector<int>> tree_labelings(const Tree& tree, const std::vector<int>& leg_spins);

bool triangle(int a2, int b2, int c2);

}  // namespace sym
