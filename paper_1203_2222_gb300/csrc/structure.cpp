// Sector tables of U(1), SU(2), fermion-parity and SU(2) x U(1) tensors (integer-exact, host).
#include "structure.h"

#include <algorithm>
#include <cstdlib>
#include <functional>

#include "../../include/symtensor.h"

namespace sym {

void fail(int code, const std::string& msg) { throw Error(code, msg); }

bool triangle(int a2, int b2, int c2) {
  return std::abs(a2 - b2) <= c2 && c2 <= a2 + b2 && ((a2 + b2 + c2) % 2 == 0);
}

Tree Tree::comb(int k) {
  Tree t;
  t.k = k;
  if (k >= 2) {
    t.nodes.push_back({0, 1});
    for (int i = 2; i < k; ++i) t.nodes.push_back({k + i - 2, i});
  }
  return t;
}

Tree Tree::comb_pair(int na, int nb) {
  Tree t;
  t.k = na + nb;
  int k = t.k;
  int top_a = na >= 1 ? 0 : -1;
  for (int i = 1; i < na; ++i) {
    t.nodes.push_back({top_a, i});
    top_a = k + (int)t.nodes.size() - 1;
  }
  int top_b = nb >= 1 ? na : -1;
  for (int i = na + 1; i < na + nb; ++i) {
    t.nodes.push_back({top_b, i});
    top_b = k + (int)t.nodes.size() - 1;
  }
  if (na >= 1 && nb >= 1) t.nodes.push_back({top_a, top_b});
  return t;
}

void Tree::validate() const {
  if (k < 0) fail(SYM_ERR_ARG, "tree: negative leg count");
  if ((int)nodes.size() != std::max(k - 1, 0)) fail(SYM_ERR_ARG, "tree: need rank-1 nodes");
  std::vector<std::array<int, 2>> rng(k + nodes.size(), {-1, -1});
  std::vector<char> used(k + nodes.size(), 0);
  for (int i = 0; i < k; ++i) rng[i] = {i, i + 1};
  for (size_t n = 0; n < nodes.size(); ++n) {
    int a = nodes[n][0], b = nodes[n][1];
    int id = k + (int)n;
    if (a < 0 || b < 0 || a >= id || b >= id) fail(SYM_ERR_ARG, "tree: child id out of range or not yet defined");
    if (used[a] || used[b] || a == b) fail(SYM_ERR_ARG, "tree: child used twice");
    if (rng[a][1] != rng[b][0]) fail(SYM_ERR_ARG, "tree: children must be adjacent leg ranges, left first");
    used[a] = used[b] = 1;
    rng[id] = {rng[a][0], rng[b][1]};
  }
  if (k >= 2 && (rng[k + nodes.size() - 1][0] != 0 || rng[k + nodes.size() - 1][1] != k))
    fail(SYM_ERR_ARG, "tree: the last node must be the root over all legs");
}

std::vector<std::vector<int>> tree_labelings(const Tree& tree, const std::vector<int>& leg_spins) {
  std::vector<std::vector<int>> out;
  int k = tree.k;
  if (k == 0) {
    out.push_back({});
    return out;
  }
  if (k == 1) {
    if (leg_spins[0] == 0) out.push_back({});
    return out;
  }
  int nn = (int)tree.nodes.size();
  std::vector<int> spin(k + nn, 0);
  for (int i = 0; i < k; ++i) spin[i] = leg_spins[i];
  std::vector<int> lab(nn - 1);
  std::function<void(int)> rec = [&](int n) {
    int a = spin[tree.nodes[n][0]], b = spin[tree.nodes[n][1]];
    if (n == nn - 1) {
      if (triangle(a, b, 0)) out.push_back(lab);
      return;
    }
    for (int c = std::abs(a - b); c <= a + b; c += 2) {
      spin[k + n] = c;
      lab[n] = c;
      rec(n + 1);
    }
  };
  rec(0);
  return out;
}

Tensor make_tensor(int group, const std::vector<Leg>& legs, int total, const Tree& tree_in) {
  if (group != SYM_U1 && group != SYM_SU2 && group != SYM_Z2F && group != SYM_SU2U1)
    fail(SYM_ERR_ARG, "unknown symmetry group");
  if (group == SYM_Z2F && total != 0 && total != 1) fail(SYM_ERR_ARG, "Z2F total parity must be 0 or 1");
  Tensor t;
  t.group = group;
  t.rank = (int)legs.size();
  if (t.rank > 6) fail(SYM_ERR_UNSUPPORTED, "rank > 6 is not supported");
  t.legs = legs;
  t.total = group == SYM_SU2 ? 0 : total;
  for (const Leg& l : legs) {
    if (l.labels.empty() || l.labels.size() != l.degens.size()) fail(SYM_ERR_ARG, "leg: empty or size mismatch");
    if (l.dir != 1 && l.dir != -1) fail(SYM_ERR_ARG, "leg: direction must be +1 or -1");
    for (size_t i = 0; i < l.labels.size(); ++i) {
      if (l.degens[i] < 1) fail(SYM_ERR_ARG, "leg: degeneracy must be >= 1");
      if (i && l.labels[i] <= l.labels[i - 1]) fail(SYM_ERR_ARG, "leg: labels must increase strictly");
      if (group == SYM_SU2 && l.labels[i] < 0) fail(SYM_ERR_ARG, "leg: negative spin");
      if (group == SYM_SU2U1 && std::abs(charge_of(group, l.labels[i])) > (1 << 20))
        fail(SYM_ERR_ARG, "leg: charge out of range");
      if (group == SYM_Z2F && l.labels[i] != 0 && l.labels[i] != 1) fail(SYM_ERR_ARG, "leg: parity must be 0 or 1");
    }
  }
  if (su2_like(group)) {
    t.tree = tree_in.k == t.rank ? tree_in : Tree::comb(t.rank);
    t.tree.validate();
    t.nin = std::max(t.rank - 2, 0);
  }
  // lexicographic product over leg positions
  std::vector<int> idx(t.rank, 0);
  t.offs.push_back(0);
  auto add = [&](const std::vector<int>& in) {
    int64_t sz = 1;
    for (int l = 0; l < t.rank; ++l) sz *= legs[l].degens[idx[l]];
    std::vector<int> key(idx);
    key.insert(key.end(), in.begin(), in.end());
    t.index.emplace(key, t.nsec());
    t.pos.insert(t.pos.end(), idx.begin(), idx.end());
    t.inner.insert(t.inner.end(), in.begin(), in.end());
    t.offs.push_back(t.offs.back() + sz);
  };
  while (true) {
    if (group == SYM_U1) {
      int64_t s = 0;
      for (int l = 0; l < t.rank; ++l) s += (int64_t)legs[l].dir * legs[l].labels[idx[l]];
      if (s == total) add({});
    } else if (group == SYM_Z2F) {  // parities add mod 2 (a direction does not change a parity)
      int s = 0;
      for (int l = 0; l < t.rank; ++l) s ^= legs[l].labels[idx[l]];
      if (s == total) add({});
    } else {
      // SU(2); SU(2) x U(1): the spins' tree labelings, where the charges obey the U(1) rule
      int64_t q = 0;
      std::vector<int> spins(t.rank);
      for (int l = 0; l < t.rank; ++l) {
        spins[l] = spin_of(group, legs[l].labels[idx[l]]);
        q += (int64_t)legs[l].dir * charge_of(group, legs[l].labels[idx[l]]);
      }
      if (q == t.total)
        for (auto& lab : tree_labelings(t.tree, spins)) add(lab);
    }
    int l = t.rank - 1;
    while (l >= 0) {
      if (++idx[l] < (int)legs[l].labels.size()) break;
      idx[l] = 0;
      --l;
    }
    if (l < 0) break;
  }
  return t;
}

}  // namespace sym
