// SU(2) recoupling: Racah 6j, F-moves, swaps and tree-transform matrices.
#include "recouple.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <unordered_map>

#include "../../include/symtensor.h"

namespace sym {

namespace {

const long double* fact_table() {
  static long double f[256];
  static std::once_flag once;
  std::call_once(once, [] {
    f[0] = 1.0L;
    for (int i = 1; i < 256; ++i) f[i] = f[i - 1] * (long double)i;
  });
  return f;
}

long double delta(int a2, int b2, int c2) {
  const long double* f = fact_table();
  return sqrtl(f[(a2 + b2 - c2) / 2] * f[(a2 - b2 + c2) / 2] * f[(-a2 + b2 + c2) / 2] /
               f[(a2 + b2 + c2) / 2 + 1]);
}

struct SixjCache {
  std::mutex mu;
  std::unordered_map<uint64_t, double> map;
};

SixjCache& cache() {
  static SixjCache c;
  return c;
}

}  // namespace

double sixj(int a, int b, int c, int d, int e, int f) {
  if (!triangle(a, b, c) || !triangle(a, e, f) || !triangle(d, b, f) || !triangle(d, e, c)) return 0.0;
  if (std::max({a, b, c, d, e, f}) > 60) fail(SYM_ERR_UNSUPPORTED, "spin too large for the 6j table");
  uint64_t key = 0;
  for (int v : {a, b, c, d, e, f}) key = key * 64 + (uint64_t)v;
  {
    std::lock_guard<std::mutex> g(cache().mu);
    auto it = cache().map.find(key);
    if (it != cache().map.end()) return it->second;
  }
  const long double* F = fact_table();
  int al[4] = {(a + b + c) / 2, (a + e + f) / 2, (d + b + f) / 2, (d + e + c) / 2};
  int be[3] = {(a + b + d + e) / 2, (b + c + e + f) / 2, (c + a + f + d) / 2};
  int tmin = *std::max_element(al, al + 4);
  int tmax = *std::min_element(be, be + 3);
  long double s = 0.0L;
  for (int t = tmin; t <= tmax; ++t) {
    long double den = F[t - al[0]] * F[t - al[1]] * F[t - al[2]] * F[t - al[3]] * F[be[0] - t] *
                      F[be[1] - t] * F[be[2] - t];
    long double term = F[t + 1] / den;
    s += (t & 1) ? -term : term;
  }
  long double v = s * delta(a, b, c) * delta(a, e, f) * delta(d, b, f) * delta(d, e, c);
  double out = (double)v;
  std::lock_guard<std::mutex> g(cache().mu);
  cache().map.emplace(key, out);
  return out;
}

double recoupF(int jd, int je, int ja, int jb, int jc, int J) {
  int ph = ja + jb + jc + J;
  if (ph % 2) return 0.0;
  double alpha = (((ph / 2) & 1) ? -1.0 : 1.0) * std::sqrt((double)(jd + 1) * (double)(je + 1));
  return alpha * sixj(ja, jb, jd, jc, J, je);
}

namespace {

using Chain = std::vector<int>;
using Expansion = std::vector<std::pair<double, Chain>>;

// A subtree in comb form: chain labels c_1..c_{m-1} (last = top) over its m
// legs, whose spins are `spins`.  Merge A and B under a node of spin c:
// |A, (B', r) f; c> = sum_g F^{g f}_{tA f' jr c} |(A, B') g, r; c>.
Expansion merge(const Chain& ca, int ta, const Chain& cb, const std::vector<int>& sb, int c) {
  Expansion out;
  size_t nb = sb.size();
  if (nb == 1) {
    Chain ch(ca);
    ch.push_back(c);
    out.emplace_back(1.0, ch);
    return out;
  }
  int f = cb.back();
  int fp = nb == 2 ? sb[0] : cb[nb - 3];
  int jr = sb.back();
  Chain cbp(cb.begin(), cb.begin() + (nb - 2));
  std::vector<int> sbp(sb.begin(), sb.end() - 1);
  for (int g = std::abs(ta - fp); g <= ta + fp; g += 2) {
    if (!triangle(g, jr, c)) continue;
    double co = recoupF(g, f, ta, fp, jr, c);
    if (co == 0.0) continue;
    for (auto& e : merge(ca, ta, cbp, sbp, g)) {
      Chain ch(e.second);
      ch.push_back(c);
      out.emplace_back(co * e.first, ch);
    }
  }
  return out;
}

// Expand the subtree `id` of a labeled tree into comb states over its legs.
Expansion comb_expand(const Tree& t, const std::vector<int>& spin, int id, std::vector<int>& leg_spins) {
  if (id < t.k) {
    leg_spins.assign(1, spin[id]);
    return Expansion{{1.0, Chain{}}};
  }
  const auto& nd = t.nodes[id - t.k];
  std::vector<int> sa, sb;
  Expansion ea = comb_expand(t, spin, nd[0], sa);
  Expansion eb = comb_expand(t, spin, nd[1], sb);
  Expansion out;
  int c = spin[id];
  for (auto& a : ea) {
    int ta = a.second.empty() ? sa[0] : a.second.back();
    for (auto& b : eb) {
      for (auto& e : merge(a.second, ta, b.second, sb, c)) out.emplace_back(a.first * b.first * e.first, e.second);
    }
  }
  leg_spins = sa;
  leg_spins.insert(leg_spins.end(), sb.begin(), sb.end());
  return out;
}

using State = std::map<Chain, double>;

State full_expand(const Tree& t, const std::vector<int>& leg_spins, const std::vector<int>& labeling) {
  int k = t.k;
  int nn = (int)t.nodes.size();
  std::vector<int> spin(k + nn, 0);
  for (int i = 0; i < k; ++i) spin[i] = leg_spins[i];
  for (int n = 0; n + 1 < nn; ++n) spin[k + n] = labeling[n];
  std::vector<int> ls;
  State st;
  for (auto& e : comb_expand(t, spin, k + nn - 1, ls)) st[e.second] += e.first;
  return st;
}

// Swap legs at positions i, i+1 of comb states whose leg spins are s.
State swap_adjacent(const State& in, const std::vector<int>& s, int i) {
  State out;
  for (auto& kv : in) {
    const Chain& e = kv.first;
    if (i == 0) {
      out[e] += kv.second * swapR(s[0], s[1], e[0]);
      continue;
    }
    int x = i == 1 ? s[0] : e[i - 2];
    int a = s[i], b = s[i + 1];
    int ei = e[i - 1], E = e[i];
    for (int ep = std::abs(x - b); ep <= x + b; ep += 2) {
      if (!triangle(ep, a, E)) continue;
      double co = 0.0;
      for (int g = std::abs(a - b); g <= a + b; g += 2) {
        if (!triangle(x, g, E)) continue;
        co += recoupF(ei, g, x, a, b, E) * swapR(a, b, g) * recoupF(ep, g, x, b, a, E);
      }
      if (co == 0.0) continue;
      Chain e2(e);
      e2[i - 1] = ep;
      out[e2] += kv.second * co;
    }
  }
  return out;
}

}  // namespace

Gamma tree_transform(const std::vector<int>& leg_spins, const Tree& tau, const std::vector<int>& perm,
                     const Tree& tau_out) {
  Gamma g;
  int k = (int)leg_spins.size();
  std::vector<int> out_spins(k);
  for (int n = 0; n < k; ++n) out_spins[n] = leg_spins[perm[n]];
  g.in_labels = tree_labelings(tau, leg_spins);
  g.out_labels = tree_labelings(tau_out, out_spins);
  size_t ni = g.in_labels.size(), no = g.out_labels.size();
  g.G.assign(no * ni, 0.0);
  if (ni == 0 || no == 0) return g;
  if (k <= 1) {
    g.G[0] = 1.0;
    return g;
  }
  std::vector<State> outexp(no);
  for (size_t o = 0; o < no; ++o) outexp[o] = full_expand(tau_out, out_spins, g.out_labels[o]);
  for (size_t i = 0; i < ni; ++i) {
    State st = full_expand(tau, leg_spins, g.in_labels[i]);
    // bubble the legs into the output order
    std::vector<int> cur(k), s(leg_spins);
    for (int n = 0; n < k; ++n) cur[n] = n;
    for (int n = 0; n < k; ++n) {
      int p = (int)(std::find(cur.begin(), cur.end(), perm[n]) - cur.begin());
      while (p > n) {
        st = swap_adjacent(st, s, p - 1);
        std::swap(cur[p - 1], cur[p]);
        std::swap(s[p - 1], s[p]);
        --p;
      }
    }
    for (size_t o = 0; o < no; ++o) {
      double acc = 0.0;
      for (auto& kv : outexp[o]) {
        auto it = st.find(kv.first);
        if (it != st.end()) acc += kv.second * it->second;
      }
      g.G[o * ni + i] = acc;
    }
  }
  return g;
}

}  // namespace sym
