// SU(2) recoupling coefficients and the tree-transform matrices Gamma.
//
// Ch. 5 "Tensor product of three irreps": two coupled bases of three spins
// are related by the recoupling coefficients F (Eq. fmove), proportional to
// Wigner 6j symbols (Eq. sixj); a swap of the two spins of one node gives the
// factor R = (-1)^(ja+jb-jc) (Eq. braid3).  Ch. 6 "Mapping between tree
// decompositions" and "Permutation of indices": the vector of a tree
// decomposition changes as v' = Gamma(tau, p, tau') v, where Gamma is a
// product of F-moves and swaps evaluated without touching the data and is
// precomputed once (Ch. 6, "Discussion on computational performance").
//
// All spins are doubled integers.  6j symbols are evaluated with Racah's
// single-sum formula; nothing here contracts Clebsch-Gordan tensors.
#pragma once

#include <vector>

#include "structure.h"

namespace sym {

// Wigner 6j {a b c; d e f} (doubled spins), 0 if a triangle fails.
double sixj(int a, int b, int c, int d, int e, int f);

// F^{jD jE}_{jA jB jC J} = (-1)^(jA+jB+jC+J) sqrt((2jD+1)(2jE+1)) {jA jB jD; jC J jE}
// = <(A,B)D, C; J | A, (B,C)E; J>  (Ch. 5, Eqs. f and sixj).
double recoupF(int jd, int je, int ja, int jb, int jc, int J);

inline double swapR(int ja, int jb, int jc) { return (((ja + jb - jc) / 2) & 1) ? -1.0 : 1.0; }

// Gamma for fixed leg spins: G[o][i] = < tau'; out labeling o | p(tau; in labeling i) >,
// where leg n of the output is leg perm[n] of the input.  Labelings are in
// the order of tree_labelings().
struct Gamma {
  std::vector<std::vector<int>> in_labels, out_labels;
  std::vector<double> G;  // out_labels.size() x in_labels.size(), row-major
};
Gamma tree_transform(const std::vector<int>& leg_spins, const Tree& tau,
                     const std::vector<int>& perm, const Tree& tau_out);

}  // namespace sym
