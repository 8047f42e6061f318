// Blockwise singular value decomposition of a symmetric tensor seen as a
// matrix (Ch. 5, "Factorization of a matrix", Eq. svd0 and svd1; Ch. 6,
// "Matrix multiplication and factorizations").
//
// The matrix is block diagonal in the fused label x of its row legs, so every
// diagonal block M_x is decomposed on its own.  The blocks are read straight
// from the tensor's blocks (each one a row-major sub-matrix of its M_x,
// because the row legs lead), so there is no separate move into matrix form.
//
// svd_jacobi_kernel: one cluster of 16 CTAs per block, one-sided Jacobi
//   (Hestenes).  A = M_x (m >= n) or M_x^T, R x C with R >= C, is copied
//   column-major into the workspace.  A sweep visits every column pair once,
//   in the round-robin order of a tournament (C - 1 rounds of C/2 disjoint
//   pairs, one warp per pair, a cluster barrier between rounds); a pair whose
//   columns are not orthogonal to within sqrt(R) ulp is rotated so that they
//   are, and the same rotation is applied to V (V = I at the start).  When a
//   whole sweep rotates nothing by more than kBigRotation(32) relative,
//   A V = W has orthogonal columns: S = their norms, U = W / S.  The sweeps
//   run first in FP32, then, from the FP32 result made orthogonal in FP64,
//   in FP64 (see the kernel).  The FP32 sweeps of blocks with at least 32
//   columns take the same pairs by column blocks, a block pair in a CTA's
//   shared memory (jacobi_sweeps_blocked).  The FP64
//   sweeps are bounded (kMaxSweeps); a block that has not converged by then
//   sets the device error word to SYM_ERR_NUMERIC.  The columns are then
//   ranked by norm (descending, ties by index) into S and a permutation.
// svd_factor_kernel: one CTA per block writes the kept singular vectors into
//   the blocks of U (row legs, bond) and V (bond, column legs), optionally
//   scaled by S.
//
// The same two kernels give the blockwise eigendecomposition of a symmetric
// tensor seen as a square matrix (Ch. 5, Eq. spectral, by blocks as the
// thesis prescribes after Eq. svd1; blocks flagged `eig`): the block is
// replaced by its symmetric part B = (M + M^T)/2 plus sigma I, where sigma is
// B's Frobenius norm (>= its spectral norm), so that B + sigma I is positive
// semidefinite.  For such a matrix the one-sided Jacobi result A V = W has
// |w_j| = lambda_j + sigma and V's columns are the eigenvectors, so the
// eigenvalues are |w_j| - sigma (absolute error ~ eps sigma, the backward
// error of any FP64 symmetric eigensolver), ranked by |lambda| descending
// (ties: the larger lambda, then the column), and U = V, V^T for the factors.
// The workspace stays L2-resident for the sizes of tensor-network bonds
// (a 300 x 300 block is 1.4 MB), so the sweeps run from L2, not HBM.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/symtensor.h"
#include "handles.h"
#include "plan.h"
#include "structure.h"

namespace cg = cooperative_groups;

namespace sym {
namespace {

constexpr int kSvdThreads = 256;
constexpr int kSvdWarps = kSvdThreads / 32;
// CTAs per diagonal block (16: a cluster size above the portable 8, allowed
// by a function attribute; two CTAs of the kernel fit on an SM)
constexpr int kSvdCluster = 16;
// dynamic shared memory a Jacobi CTA may take for the FP32 sweeps by column
// blocks (two CTAs of 256 threads and 128 registers share an SM)
constexpr int kSvdSmem32Max = 100 * 1024;
constexpr int kMaxSweeps = 64;    // FP64 sweeps before a block counts as not converged
constexpr int kMaxSweeps32 = 40;  // FP32 sweeps (their result only seeds the FP64 ones)
// An FP64 sweep whose rotations all had |w_p.w_q| <= kBigRotation |w_p| |w_q|
// ends the sweeps: what it leaves is of order kBigRotation^2 from the pairs'
// coupling plus the rotation's own residual (the angle is formed to FP32
// accuracy, about 6e-8 of kBigRotation), both near the FP64 rounding level,
// so a further sweep would find nothing to rotate.
constexpr double kBigRotation = 1e-8;
// The FP32 sweeps stop on the same rule at 1e-4: what they leave (1e-8) is
// below FP32's own rounding of the pair products.
constexpr float kBigRotation32 = 1e-4f;

struct SvdBlock {
  int m, n;    // M_x is m x n
  int R, C;    // working matrix A (R x C, R >= C): M_x, or M_x^T when trans
  int trans;   // A = M_x^T (m < n)
  int keep;    // singular vectors the factor kernel writes
  int t0, nt;  // pieces of T
  int u0, nu;  // pieces of U
  int v0, nv;  // pieces of V
  int slot;    // position of the block in ascending x
  int ks;      // first kept singular value of the block in the bond order
  double vscale;  // SU(2): sqrt(2j+1) (the factors carry it, S is divided by it), else 1
  int eig;        // eigendecomposition of the symmetric part (square block) instead of the SVD
  double sgn;     // eig, SU(2) with an incoming row leg: (-1)^{2j}, the sign of the dense block; else 1
  int bw;         // FP32 sweeps by column blocks of bw columns (0: by column pairs)
  int bw64;       // the same for the FP64 sweeps
  int64_t w;   // workspace offset: W (R x C, column-major), V (C x C), norms (C), sorted S (C), then
               // the Jacobi kernel's A (R x C), Newton-Schulz factor (C x C), FP32 W and V
  int64_t s;   // first singular value of the block in S and in the permutation
};

// A tensor block inside its M_x: rows r0.., columns c0.. (row-major, rows x cols).
struct SvdPiece {
  int64_t off;
  int r0, c0, rows, cols;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  // xor butterfly: every lane ends with the same sum (each step adds the same
  // two values on both partners)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The Jacobi angle of a column pair (p, q) with a = |w_p|^2, bb = |w_q|^2,
// g = w_p.w_q: if the pair is not orthogonal to within tol, the rotation by
// t = tan(theta), the smaller root of t^2 + 2 zeta t - 1 = 0 with
// zeta = (bb - a) / (2 g), makes it so.  Every lane takes the same decision
// (identical butterfly sums).
template <typename T>
struct JacobiArith;

template <>
struct JacobiArith<float> {
  static constexpr float kEps = FLT_EPSILON;
  static __device__ __forceinline__ bool angle(float a, float bb, float g, float sab, float tol, float& c,
                                               float& s) {
    if (!(fabsf(g) > tol * sab)) return false;
    const float zeta = (bb - a) / (2.0f * g);
    const float t = fabsf(zeta) > 1e18f ? 0.5f / zeta
                                        : copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = c * t;
    return true;
  }
};

template <>
struct JacobiArith<double> {
  static constexpr double kEps = DBL_EPSILON;
  // The angle itself needs only FP32 accuracy: an inexact angle is still an
  // exact rotation (c^2 + s^2 = 1 to FP64 precision), it just leaves the
  // pair slightly non-orthogonal for the next sweep.  So t = sign(d) h /
  // (|d| + sqrt(d^2 + h^2)) (d = bb - a, h = 2 g; the same root) is formed in
  // FP32 after scaling d and h by a power of two, and c = (1 + t^2)^(-1/2)
  // by two Newton steps in FP64 from the FP32 estimate -- GB300's FP64 units
  // are few, and FP64 square roots and divisions cost many of their cycles.
  static __device__ __forceinline__ bool angle(double a, double bb, double g, double sab, double tol, double& c,
                                               double& s) {
    if (!(fabs(g) > tol * sab)) return false;
    const double d = bb - a, h = 2.0 * g;
    const double m = fmax(fabs(d), fabs(h));
    const int ex = (__double2hiint(m) >> 20) & 0x7ff;  // biased exponent of m
    float tf = 0.0f;
    if (ex > 0 && ex < 2046) {
      const double sc = __hiloint2double((2046 - ex) << 20, 0);  // 2^(1023 - e): m * sc in [1, 2)
      const float df = (float)(d * sc), hf = (float)(h * sc);
      tf = copysignf(1.0f, df) * hf / (fabsf(df) + sqrtf(fmaf(df, df, hf * hf)));
    }
    double t;
    if (tf != 0.0f && isfinite(tf)) {
      t = (double)tf;
    } else {  // out of FP32's reach: the angle in FP64
      const double zeta = d / h;
      t = fabs(zeta) > 1e150 ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
    }
    const double x = fma(t, t, 1.0);
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x * y, y, 1.5);  // Newton steps for x^(-1/2): y (3 - x y^2) / 2
    y = y * fma(-0.5 * x * y, y, 1.5);
    c = y;
    s = y * t;
    return true;
  }
};

// Rotate one column pair (p, q) of W (length R) and V (length C) if needed.
// NR rows per lane held in registers (R <= 32 NR); V's columns are loaded
// with W's, so a pair costs one round trip to L2.
template <typename T, int NR>
// With na, nb (the pair's squared column norms, carried as in
// rotate_pair_smem below) one dot product a pair instead of three.
__device__ __forceinline__ int rotate_pair(T* wp, T* wq, T* vp, T* vq, T* na, T* nb, int R, int C, int lane, T tol,
                                           T big) {
  T xw[NR], yw[NR], xv[NR], yv[NR];
  T a = 0, bb = 0;
  if (na) {
    a = __ldcg(na);
    bb = __ldcg(nb);
  }
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    const int i = lane + 32 * u;
    xw[u] = i < R ? __ldcg(wp + i) : T(0);
    yw[u] = i < R ? __ldcg(wq + i) : T(0);
    xv[u] = i < C ? __ldcg(vp + i) : T(0);
    yv[u] = i < C ? __ldcg(vq + i) : T(0);
  }
  T g = 0;
  if (!na) {
#pragma unroll
    for (int u = 0; u < NR; ++u) {
      a = fma(xw[u], xw[u], a);
      bb = fma(yw[u], yw[u], bb);
    }
    a = warp_sum(a);
    bb = warp_sum(bb);
  }
#pragma unroll
  for (int u = 0; u < NR; ++u) g = fma(xw[u], yw[u], g);
  g = warp_sum(g);
  const T sab = sqrt(a * bb);
  T c, s;
  if (!JacobiArith<T>::angle(a, bb, g, sab, tol, c, s)) return 0;
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    const int i = lane + 32 * u;
    if (i < R) {
      __stcg(wp + i, c * xw[u] - s * yw[u]);
      __stcg(wq + i, s * xw[u] + c * yw[u]);
    }
    if (i < C) {
      __stcg(vp + i, c * xv[u] - s * yv[u]);
      __stcg(vq + i, s * xv[u] + c * yv[u]);
    }
  }
  if (na && lane == 0) {
    const T cs2g = T(2) * c * s * g, cc = c * c, ss = s * s;
    __stcg(na, fma(cc, a, fma(ss, bb, -cs2g)));
    __stcg(nb, fma(ss, a, fma(cc, bb, cs2g)));
  }
  return fabs(g) > big * sab ? 2 : 1;
}

// Any R: the columns streamed twice (products, then the rotation).
template <typename T>
__device__ __noinline__ int rotate_pair_stream(T* wp, T* wq, T* vp, T* vq, int R, int C, int lane, T tol, T big) {
  T a = 0, bb = 0, g = 0;
  for (int i = lane; i < R; i += 32) {
    const T x = __ldcg(wp + i), y = __ldcg(wq + i);
    a = fma(x, x, a);
    bb = fma(y, y, bb);
    g = fma(x, y, g);
  }
  a = warp_sum(a);
  bb = warp_sum(bb);
  g = warp_sum(g);
  const T sab = sqrt(a * bb);
  T c, s;
  if (!JacobiArith<T>::angle(a, bb, g, sab, tol, c, s)) return 0;
  for (int i = lane; i < R; i += 32) {
    const T x = __ldcg(wp + i), y = __ldcg(wq + i);
    __stcg(wp + i, c * x - s * y);
    __stcg(wq + i, s * x + c * y);
  }
  for (int i = lane; i < C; i += 32) {
    const T x = __ldcg(vp + i), y = __ldcg(vq + i);
    __stcg(vp + i, c * x - s * y);
    __stcg(vq + i, s * x + c * y);
  }
  return fabs(g) > big * sab ? 2 : 1;
}

// Per-cluster state of the sweeps (shared memory of every CTA; rank 0's
// flags are the cluster's).
struct SweepCtl {
  int flag[2];
  int any;
};

// Sweeps of one-sided Jacobi on (W, V), at most max_sweeps; returns the
// sweeps taken, conv = the last sweep rotated nothing.  The C/2 pairs of a
// round (tournament order, an odd C playing against a bye) go to the
// cluster's warps; cluster barriers separate the rounds.
template <typename T>
__device__ int jacobi_sweeps(T* W, T* V, T* nrm2, int R, int C, int max_sweeps, T tol, cg::cluster_group& cluster,
                             SweepCtl* ctl, int* flag0, int crank, int cw, int lane, int& gsweep,
                             unsigned long long& myrot, bool& conv, T big_tol) {
  constexpr int kCW = kSvdCluster * kSvdWarps;
  const int Ce = C + (C & 1);
  const int rpl = (R + 31) / 32;
  const int nr = rpl <= 1 ? 1 : rpl <= 2 ? 2 : rpl <= 4 ? 4 : rpl <= 8 ? 8 : rpl <= 9 ? 9 : rpl <= 12 ? 12 : 0;
  int sweeps = 0;
  conv = C < 2;
  while (!conv && sweeps < max_sweeps) {
    ++sweeps;
    const int gs = ++gsweep;  // sweeps so far over both precisions (same in every thread): picks the flag
    int did = 0, big = 0;
    if (nrm2 && nr) {  // the squared column norms, exact at the sweep's start, carried by the rotations
      for (int j = cw; j < C; j += kCW) {
        const T* wj = W + (int64_t)j * R;
        T a = 0;
        for (int i = lane; i < R; i += 32) {
          const T x = __ldcg(wj + i);
          a = fma(x, x, a);
        }
        a = warp_sum(a);
        if (lane == 0) __stcg(nrm2 + j, a);
      }
      cluster.sync();
    }
    T* const carry = nr ? nrm2 : nullptr;
    for (int r = 0; r < Ce - 1; ++r) {
      for (int k = cw; k < Ce / 2; k += kCW) {
        int p = k == 0 ? r : (r + k) % (Ce - 1);
        int q = k == 0 ? Ce - 1 : (r - k + Ce - 1) % (Ce - 1);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= C) continue;
        T* wp = W + (int64_t)p * R;
        T* wq = W + (int64_t)q * R;
        T* vp = V + (int64_t)p * C;
        T* vq = V + (int64_t)q * C;
        int rot;
        T* na = carry ? carry + p : nullptr;
        T* nb = carry ? carry + q : nullptr;
        switch (nr) {
          case 1: rot = rotate_pair<T, 1>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol); break;
          case 2: rot = rotate_pair<T, 2>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol); break;
          case 4: rot = rotate_pair<T, 4>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol); break;
          case 8: rot = rotate_pair<T, 8>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol); break;
          case 9: rot = rotate_pair<T, 9>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol); break;
          case 12: rot = rotate_pair<T, 12>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol); break;
          default: rot = rotate_pair_stream<T>(wp, wq, vp, vq, R, C, lane, tol, big_tol); break;
        }
        if (rot) {
          did = 1;
          big |= rot == 2;
          ++myrot;
        }
      }
      cluster.sync();  // the next round's pairs read columns this round wrote
    }
    // did any warp of the cluster rotate?  flags alternate between sweeps, so
    // the one read now is never the one being cleared for the next sweep
    const int f = (__syncthreads_or(did) ? 1 : 0) | (__syncthreads_or(big) ? 2 : 0);
    if (f && threadIdx.x == 0) atomicOr(flag0 + (gs & 1), f);
    cluster.sync();
    if (threadIdx.x == 0) {
      ctl->any = flag0[gs & 1];
      if (crank == 0) ctl->flag[(gs + 1) & 1] = 0;
    }
    __syncthreads();
    // converged: nothing rotated by more than big_tol relative -- what
    // remains is then of order big_tol^2
    conv = !(ctl->any & 2);
    __syncthreads();  // any and gsweep are rewritten by the next sweep
  }
  return sweeps;
}

// Rotate one column pair of W (length R) and V (length C) held in shared
// memory; NR rows per lane.  The squared column norms *na, *nb are carried
// from rotation to rotation (recomputed at every sweep's start), so a pair
// costs one dot product (w_p . w_q), not three; the rotation updates them
// exactly as it rotates the columns: |w_p'|^2 = c^2 a - 2 c s g + s^2 b,
// |w_q'|^2 = s^2 a + 2 c s g + c^2 b.  Returns 0 (no rotation), 1, or 2 (a
// rotation larger than big relative to the pair's norms).
template <typename T, int NR>
__device__ __forceinline__ int rotate_pair_smem(T* wp, T* wq, T* vp, T* vq, T* na, T* nb, int R, int C, int lane,
                                                T tol, T big) {
  T xw[NR], yw[NR];
  T g = 0;
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    const int i = lane + 32 * u;
    xw[u] = i < R ? wp[i] : T(0);
    yw[u] = i < R ? wq[i] : T(0);
    g = fma(xw[u], yw[u], g);
  }
  g = warp_sum(g);
  const T a = *na, bb = *nb;
  const T sab = sqrt(a * bb);
  T c, sn;
  if (!JacobiArith<T>::angle(a, bb, g, sab, tol, c, sn)) return 0;
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    const int i = lane + 32 * u;
    if (i < R) {
      wp[i] = c * xw[u] - sn * yw[u];
      wq[i] = sn * xw[u] + c * yw[u];
    }
    if (i < C) {
      const T x = vp[i], y = vq[i];
      vp[i] = c * x - sn * y;
      vq[i] = sn * x + c * y;
    }
  }
  const T cs2g = T(2) * c * sn * g, cc = c * c, ss = sn * sn;
  __syncwarp();  // every lane has read the old norms
  if (lane == 0) {
    *na = fma(cc, a, fma(ss, bb, -cs2g));
    *nb = fma(ss, a, fma(cc, bb, cs2g));
  }
  return fabs(g) > big * sab ? 2 : 1;
}

// FP32 sweeps by column blocks: the C columns form kColBlocks blocks of bw
// (the last ones ragged or empty), and a sweep is the tournament over the
// blocks (kColBlocks - 1 rounds of kSvdCluster disjoint block pairs).  In a
// round, CTA k of the cluster takes block pair k -- the columns of W and V
// -- into its shared memory, rotates every cross pair (p in P, q in Q; in
// the first round also the pairs inside P and inside Q) in bw inner rounds
// of disjoint pairs separated by CTA barriers, and writes the columns back;
// a cluster barrier separates the rounds.  Every column pair is visited once
// a sweep, as in the order by pairs, but a sweep needs kColBlocks - 1 cluster
// barriers instead of C - 1, and the pairs' columns come from shared memory.
constexpr int kColBlocks = 2 * kSvdCluster;
template <typename T, int NR>
__device__ int jacobi_sweeps_blocked(T* W, T* V, T* nrm2, int R, int C, int bw, int max_sweeps, T tol,
                                     cg::cluster_group& cluster, SweepCtl* ctl, int* flag0, int crank, int lane,
                                     int& gsweep, unsigned long long& myrot, bool& conv, T big_tol, T* sm) {
  const int warp = threadIdx.x >> 5;
  constexpr int kCW = kSvdCluster * kSvdWarps;
  const int cw = crank * kSvdWarps + warp;
  T* Wp = sm;  // bw columns of R, then Q's, then V's columns of P and Q (C each), then their squared norms
  T* Wq = Wp + (int64_t)bw * R;
  T* Vp = Wq + (int64_t)bw * R;
  T* Vq = Vp + (int64_t)bw * C;
  T* Np = Vq + (int64_t)bw * C;
  T* Nq = Np + bw;
  const int bwe = bw + (bw & 1);  // a block's own tournament: bwe - 1 rounds of bwe / 2 pairs
  int sweeps = 0;
  conv = C < 2;
  while (!conv && sweeps < max_sweeps) {
    ++sweeps;
    const int gs = ++gsweep;
    int did = 0, big = 0;
    for (int j = cw; j < C; j += kCW) {  // the squared column norms, exact at the sweep's start
      const T* wj = W + (int64_t)j * R;
      T a = 0;
      for (int i = lane; i < R; i += 32) {
        const T x = __ldcg(wj + i);
        a = fma(x, x, a);
      }
      a = warp_sum(a);
      if (lane == 0) __stcg(nrm2 + j, a);
    }
    cluster.sync();
    auto rot = [&](T* wp, T* wq, T* vp, T* vq, T* na, T* nb) {
      const int r = rotate_pair_smem<T, NR>(wp, wq, vp, vq, na, nb, R, C, lane, tol, big_tol);
      if (r) {
        did = 1;
        big |= r == 2;
        ++myrot;
      }
    };
    for (int r = 0; r < kColBlocks - 1; ++r) {
      const int k = crank;
      const int P = k == 0 ? r : (r + k) % (kColBlocks - 1);
      const int Q = k == 0 ? kColBlocks - 1 : (r - k + kColBlocks - 1) % (kColBlocks - 1);
      const int p0 = P * bw, np = max(0, min(bw, C - p0));
      const int q0 = Q * bw, nq = max(0, min(bw, C - q0));
      // the two blocks' columns are contiguous in the column-major W and V
      for (int i = threadIdx.x; i < np * R; i += kSvdThreads) Wp[i] = __ldcg(W + (int64_t)p0 * R + i);
      for (int i = threadIdx.x; i < nq * R; i += kSvdThreads) Wq[i] = __ldcg(W + (int64_t)q0 * R + i);
      for (int i = threadIdx.x; i < np * C; i += kSvdThreads) Vp[i] = __ldcg(V + (int64_t)p0 * C + i);
      for (int i = threadIdx.x; i < nq * C; i += kSvdThreads) Vq[i] = __ldcg(V + (int64_t)q0 * C + i);
      for (int i = threadIdx.x; i < np; i += kSvdThreads) Np[i] = __ldcg(nrm2 + p0 + i);
      for (int i = threadIdx.x; i < nq; i += kSvdThreads) Nq[i] = __ldcg(nrm2 + q0 + i);
      __syncthreads();
      if (r == 0) {  // the pairs inside P and inside Q: each block's own tournament, side by side
        for (int ir = 0; ir < bwe - 1; ++ir) {
          for (int t = warp; t < bwe; t += kSvdWarps) {
            const int side = t < bwe / 2 ? 0 : 1, kk = side ? t - bwe / 2 : t;
            int a = kk == 0 ? ir : (ir + kk) % (bwe - 1);
            int c = kk == 0 ? bwe - 1 : (ir - kk + bwe - 1) % (bwe - 1);
            const int n = side ? nq : np;
            if (a < n && c < n) {
              T* w0 = side ? Wq : Wp;
              T* v0 = side ? Vq : Vp;
              T* n0 = side ? Nq : Np;
              rot(w0 + (int64_t)a * R, w0 + (int64_t)c * R, v0 + (int64_t)a * C, v0 + (int64_t)c * C, n0 + a, n0 + c);
            }
          }
          __syncthreads();
        }
      }
      for (int ir = 0; ir < bw; ++ir) {  // the cross pairs (i, (i + ir) mod bw)
        for (int i = warp; i < bw; i += kSvdWarps) {
          const int j = (i + ir) % bw;
          if (i < np && j < nq)
            rot(Wp + (int64_t)i * R, Wq + (int64_t)j * R, Vp + (int64_t)i * C, Vq + (int64_t)j * C, Np + i, Nq + j);
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < np * R; i += kSvdThreads) __stcg(W + (int64_t)p0 * R + i, Wp[i]);
      for (int i = threadIdx.x; i < nq * R; i += kSvdThreads) __stcg(W + (int64_t)q0 * R + i, Wq[i]);
      for (int i = threadIdx.x; i < np * C; i += kSvdThreads) __stcg(V + (int64_t)p0 * C + i, Vp[i]);
      for (int i = threadIdx.x; i < nq * C; i += kSvdThreads) __stcg(V + (int64_t)q0 * C + i, Vq[i]);
      for (int i = threadIdx.x; i < np; i += kSvdThreads) __stcg(nrm2 + p0 + i, Np[i]);
      for (int i = threadIdx.x; i < nq; i += kSvdThreads) __stcg(nrm2 + q0 + i, Nq[i]);
      cluster.sync();  // the next round reads columns this round wrote, on other CTAs
    }
    const int f = (__syncthreads_or(did) ? 1 : 0) | (__syncthreads_or(big) ? 2 : 0);
    if (f && threadIdx.x == 0) atomicOr(flag0 + (gs & 1), f);
    cluster.sync();
    if (threadIdx.x == 0) {
      ctl->any = flag0[gs & 1];
      if (crank == 0) ctl->flag[(gs + 1) & 1] = 0;
    }
    __syncthreads();
    conv = !(ctl->any & 2);
    __syncthreads();
  }
  return sweeps;
}

// out[:, j] = scale * sum_i X[i, j] Aop[:, i]  (column-major: Aop rows x C,
// X C x C, out rows x C); a warp per (column j, 128 rows).
__device__ void gemm_cols(const double* Aop, int rows, int C, const double* X, double* out, double scale, int cw,
                          int lane) {
  constexpr int kCW = kSvdCluster * kSvdWarps;
  const int nrb = (rows + 127) / 128;
  for (int task = cw; task < C * nrb; task += kCW) {
    const int j = task / nrb, r0 = (task - j * nrb) * 128;
    const double* xj = X + (int64_t)j * C;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int i = 0; i < C; ++i) {
      const double x = __ldcg(xj + i);
      const double* ai = Aop + (int64_t)i * rows;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + lane + 32 * u;
        if (r < rows) acc[u] = fma(x, __ldcg(ai + r), acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + lane + 32 * u;
      if (r < rows) __stcg(out + (int64_t)j * rows + r, scale * acc[u]);
    }
  }
}

// G = 1.5 I - 0.5 Q^T Q (Q: C x C column-major), the factor of one
// Newton-Schulz step Q <- Q G towards the orthogonal polar factor of Q; a
// warp per (row i, four columns j).
__device__ void newton_schulz_factor(const double* Q, int C, double* G, int cw, int lane) {
  constexpr int kCW = kSvdCluster * kSvdWarps;
  const int nj = (C + 3) / 4;
  for (int task = cw; task < C * nj; task += kCW) {
    const int i = task / nj, j0 = (task - i * nj) * 4;
    const double* qi = Q + (int64_t)i * C;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = lane; k < C; k += 32) {
      const double x = __ldcg(qi + k);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u < C) acc[u] = fma(x, __ldcg(Q + (int64_t)(j0 + u) * C + k), acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double v = warp_sum(acc[u]);
      if (lane == 0 && j0 + u < C) __stcg(G + i + (int64_t)(j0 + u) * C, (i == j0 + u ? 1.5 : 0.0) - 0.5 * v);
    }
  }
}

// One cluster of kSvdCluster CTAs per block: the pairs of a round are spread
// over the cluster's warps and the rounds are separated by cluster barriers
// (their release / acquire order the workspace writes; the workspace is read
// and written at L2, bypassing L1, so no SM keeps a stale copy).
//
// Mixed precision.  GB300 runs FP32 at many times its FP64 rate, so the
// sweeps that do most of the work run in FP32 on A scaled by a power of two
// (max |A| in [1/2, 1): no FP32 overflow or underflow of the bulk); their V
// is made orthogonal to FP64 precision by two Newton-Schulz steps in FP64
// (an orthogonality error e becomes ~1.5 e^2 per step), W = A V is formed in
// FP64, and FP64 sweeps polish W and V to FP64 convergence.  The result is
// the FP64 Jacobi result; the FP32 part only chooses the starting point.
__global__ void __cluster_dims__(kSvdCluster, 1, 1) __launch_bounds__(kSvdThreads, 2)
    svd_jacobi_kernel(const SvdBlock* __restrict__ blocks, const SvdPiece* __restrict__ pieces,
                      const double* __restrict__ T, double* __restrict__ work, double* __restrict__ S,
                      int* __restrict__ perm, int* __restrict__ sweeps, long long* __restrict__ rotations,
                      int* __restrict__ err) {
  __shared__ unsigned long long nrot[2];
  __shared__ unsigned long long amax;
  __shared__ SweepCtl ctl;
  __shared__ double wsum[kSvdWarps];
  __shared__ double fpart;  // eig: this CTA's part of the squared Frobenius norm
  extern __shared__ double sm_pair[];  // the sweeps by column blocks: a block pair of W and V
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const SvdBlock b = blocks[blockIdx.x / kSvdCluster];
  const int R = b.R, C = b.C;
  const int64_t RC = (int64_t)R * C, CC = (int64_t)C * C;
  double* W = work + b.w;  // FP64 W, then V, norms, sorted S (the factor kernel's view)
  double* V = W + RC;
  double* nrm = V + CC;
  double* Ss = nrm + C;
  double* A = Ss + C;  // FP64 A (scaled), the Newton-Schulz factor, FP32 W and V
  double* G = A + RC;
  float* W32 = reinterpret_cast<float*>(G + CC);
  float* V32 = W32 + RC;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ct = crank * kSvdThreads + tid;       // thread of the cluster
  const int cw = crank * kSvdWarps + (tid >> 5);  // warp of the cluster
  constexpr int kCT = kSvdCluster * kSvdThreads;
  if (tid == 0) {
    nrot[0] = nrot[1] = 0;
    amax = 0;
    ctl.flag[0] = ctl.flag[1] = 0;
    ctl.any = 0;
  }
  cluster.sync();  // shared state initialised before any remote access

  // A (m >= n: M_x, else M_x^T) in FP64, column-major, and max |A|
  for (int64_t i = ct; i < RC; i += kCT) __stcg(A + i, 0.0);
  cluster.sync();
  unsigned long long mx = 0;
  for (int k = 0; k < b.nt; ++k) {
    const SvdPiece pc = pieces[b.t0 + k];
    const int64_t n = (int64_t)pc.rows * pc.cols;
    for (int64_t e = ct; e < n; e += kCT) {
      const int i = (int)(e / pc.cols), j = (int)(e - (int64_t)i * pc.cols);
      const int64_t r = pc.r0 + i, c = pc.c0 + j;
      const double v = T[pc.off + e];
      __stcg(b.trans ? A + c + r * R : A + r + c * R, v);
      mx = max(mx, (unsigned long long)__double_as_longlong(fabs(v)));  // |v| >= 0 orders as its bits
    }
  }
  double shift = 0.0;  // eig: sigma
  if (b.eig) {
    cluster.sync();  // the whole block is in A
    // the symmetric part, in place (the thread of (r, c), r < c, writes both
    // halves), and its squared Frobenius norm
    double f2 = 0.0;
    for (int64_t e = ct; e < RC; e += kCT) {
      const int r = (int)(e % R), c = (int)(e / R);
      if (r < c) {
        const int64_t t = c + (int64_t)r * R;
        const double v = 0.5 * (__ldcg(A + e) + __ldcg(A + t));
        __stcg(A + e, v);
        __stcg(A + t, v);
        f2 = fma(2.0 * v, v, f2);
      } else if (r == c) {
        const double v = __ldcg(A + e);
        f2 = fma(v, v, f2);
      }
    }
    f2 = warp_sum(f2);
    if (lane == 0) wsum[tid >> 5] = f2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kSvdWarps; ++w) t += wsum[w];
      fpart = t;
    }
    cluster.sync();  // every CTA's part and the symmetric part are written
    double tot = 0.0;  // the same sum, in the same order, in every thread
    for (int r = 0; r < kSvdCluster; ++r) tot += *cluster.map_shared_rank(&fpart, r);
    shift = sqrt(tot);
    for (int j = ct; j < C; j += kCT) __stcg(A + j + (int64_t)j * R, __ldcg(A + j + (int64_t)j * R) + shift);
    cluster.sync();
    mx = 0;
    for (int64_t e = ct; e < RC; e += kCT)
      mx = max(mx, (unsigned long long)__double_as_longlong(fabs(__ldcg(A + e))));
  }
  if (mx) atomicMax(cluster.map_shared_rank(&amax, 0), mx);
  cluster.sync();
  const double amx = __longlong_as_double((long long)*cluster.map_shared_rank(&amax, 0));
  // scale sa = 2^-e with 2^e <= max |A| < 2^(e+1); 1 for a zero or non-finite block
  const int ex = (__double2hiint(amx) >> 20) & 0x7ff;
  const bool scaled = ex > 0 && ex < 2046;
  const double sa = scaled ? __hiloint2double((2046 - ex) << 20, 0) : 1.0;
  const double unsa = scaled ? __hiloint2double(ex << 20, 0) : 1.0;  // 1 / sa

  for (int64_t i = ct; i < RC; i += kCT) __stcg(W32 + i, (float)(sa * __ldcg(A + i)));
  for (int64_t i = ct; i < CC; i += kCT) __stcg(V32 + i, (i % (C + 1) == 0) ? 1.0f : 0.0f);
  cluster.sync();

  int* flag0 = cluster.map_shared_rank(ctl.flag, 0);
  unsigned long long rot32 = 0, rot64 = 0;
  bool conv32, conv;
  int gsweep = 0;
  const float tol32 = sqrtf((float)R) * FLT_EPSILON;
  int sw32;
  switch (b.bw ? (R + 31) / 32 : 0) {
#define SYM_BLOCKED(NR)                                                                                           \
  case NR:                                                                                                         \
    sw32 = jacobi_sweeps_blocked<float, NR>(W32, V32, reinterpret_cast<float*>(nrm), R, C, b.bw, kMaxSweeps32,     \
                                            tol32, cluster, &ctl, flag0, crank, lane, gsweep, rot32, conv32,       \
                                            kBigRotation32, reinterpret_cast<float*>(sm_pair));                    \
    break;
    SYM_BLOCKED(1)
    SYM_BLOCKED(2)
    SYM_BLOCKED(3)
    SYM_BLOCKED(4)
    SYM_BLOCKED(5)
    SYM_BLOCKED(6)
    SYM_BLOCKED(7)
    SYM_BLOCKED(8)
    SYM_BLOCKED(9)
    SYM_BLOCKED(10)
    SYM_BLOCKED(11)
    SYM_BLOCKED(12)
#undef SYM_BLOCKED
    default:
      sw32 = jacobi_sweeps<float>(W32, V32, reinterpret_cast<float*>(nrm), R, C, kMaxSweeps32, tol32, cluster, &ctl,
                                  flag0, crank, cw, lane, gsweep, rot32, conv32, kBigRotation32);
  }

  // V = V32 made orthogonal in FP64: two Newton-Schulz steps through the G
  // buffer, the first one's product in W's buffer (free until W = A V)
  for (int64_t i = ct; i < CC; i += kCT) __stcg(V + i, (double)__ldcg(V32 + i));
  cluster.sync();
  newton_schulz_factor(V, C, G, cw, lane);
  cluster.sync();
  gemm_cols(V, C, C, G, W, 1.0, cw, lane);
  cluster.sync();
  newton_schulz_factor(W, C, G, cw, lane);
  cluster.sync();
  gemm_cols(W, C, C, G, V, 1.0, cw, lane);
  cluster.sync();
  gemm_cols(A, R, C, V, W, sa, cw, lane);  // W = (sa A) V
  cluster.sync();

  const double tol64 = sqrt((double)R) * DBL_EPSILON;
  int sw64;
  switch (b.bw64 ? (R + 31) / 32 : 0) {
#define SYM_BLOCKED(NR)                                                                                          \
  case NR:                                                                                                        \
    sw64 = jacobi_sweeps_blocked<double, NR>(W, V, nrm, R, C, b.bw64, kMaxSweeps, tol64, cluster, &ctl, flag0,   \
                                             crank, lane, gsweep, rot64, conv, kBigRotation, sm_pair);          \
    break;
    SYM_BLOCKED(1)
    SYM_BLOCKED(2)
    SYM_BLOCKED(3)
    SYM_BLOCKED(4)
    SYM_BLOCKED(5)
    SYM_BLOCKED(6)
    SYM_BLOCKED(7)
    SYM_BLOCKED(8)
    SYM_BLOCKED(9)
    SYM_BLOCKED(10)
    SYM_BLOCKED(11)
    SYM_BLOCKED(12)
#undef SYM_BLOCKED
    default:
      sw64 = jacobi_sweeps<double>(W, V, nrm, R, C, kMaxSweeps, tol64, cluster, &ctl, flag0, crank, cw, lane, gsweep,
                                   rot64, conv, kBigRotation);
  }
  if (lane == 0 && rot32) atomicAdd(cluster.map_shared_rank(&nrot[0], 0), rot32);
  if (lane == 0 && rot64) atomicAdd(cluster.map_shared_rank(&nrot[1], 0), rot64);

  // undo the scaling (a power of two: exact) and take the column norms
  constexpr int kCW = kSvdCluster * kSvdWarps;
  for (int j = cw; j < C; j += kCW) {
    double* wj = W + (int64_t)j * R;
    double a = 0.0;
    for (int i = lane; i < R; i += 32) {
      const double x = unsa * __ldcg(wj + i);
      __stcg(wj + i, x);
      a = fma(x, x, a);
    }
    a = warp_sum(a);
    if (lane == 0) __stcg(nrm + j, sqrt(a));
  }
  cluster.sync();  // norms written; the rotation counts have arrived at rank 0
  if (crank == 0 && tid == 0) {
    if (!conv) atomicExch(err, SYM_ERR_NUMERIC);
    sweeps[2 * b.slot] = sw64;
    sweeps[2 * b.slot + 1] = sw32;
    rotations[2 * b.slot] = (long long)nrot[1];
    rotations[2 * b.slot + 1] = (long long)nrot[0];
  }
  for (int j = ct; j < C; j += kCT) {
    const double v = __ldcg(nrm + j);
    int rank = 0;
    if (!b.eig) {
      for (int i = 0; i < C; ++i) {
        const double u = __ldcg(nrm + i);
        rank += (u > v) || (u == v && i < j);
      }
      S[b.s + rank] = v / b.vscale;
      Ss[rank] = v;
    } else {  // lambda = |w| - sigma, ranked by |lambda| (ties: larger lambda, then column)
      const double lj = v - shift, aj = fabs(lj);
      for (int i = 0; i < C; ++i) {
        const double li = __ldcg(nrm + i) - shift, ai = fabs(li);
        rank += (ai > aj) || (ai == aj && (li > lj || (li == lj && i < j)));
      }
      S[b.s + rank] = b.sgn * lj / b.vscale;
      Ss[rank] = lj;
    }
    perm[b.s + rank] = j;
  }
}

// From A V = W with orthogonal columns: M = (W / S) diag(S) V^T when A = M,
// and M = V diag(S) (W / S)^T when A = M^T.
__global__ void __launch_bounds__(kSvdThreads)
    svd_factor_kernel(const SvdBlock* __restrict__ blocks, const SvdPiece* __restrict__ pieces,
                      const double* __restrict__ work, const int* __restrict__ perm, double* __restrict__ U,
                      double* __restrict__ Vt, double* __restrict__ Sk, int absorb) {
  const SvdBlock b = blocks[blockIdx.x];
  const int R = b.R, C = b.C, k = b.keep;
  if (k == 0) return;
  const double* W = work + b.w;
  const double* V = W + (int64_t)R * C;
  const double* Ss = V + (int64_t)C * C + C;
  const int* pm = perm + b.s;
  const int tid = threadIdx.x;
  // SU(2): the factors are vscale times the orthonormal ones and the values
  // are divided by it; absorbing S gives the orthonormal factor times sigma
  const double vs = b.vscale;
  if (b.eig) {  // M = Q diag(lambda) Q^T: U = vs Q, V = sgn vs Q^T, values sgn lambda / vs
    const double sg = b.sgn;
    if (Sk)
      for (int j = tid; j < k; j += kSvdThreads) Sk[b.ks + j] = sg * Ss[j] / vs;
    for (int q = 0; q < b.nu; ++q) {
      const SvdPiece pc = pieces[b.u0 + q];
      const int64_t n = (int64_t)pc.rows * k;
      for (int64_t e = tid; e < n; e += kSvdThreads) {
        const int i = (int)(e / k), j = (int)(e - (int64_t)i * k);
        U[pc.off + e] = V[pc.r0 + i + (int64_t)pm[j] * C] * (absorb == 1 ? sg * Ss[j] : vs);
      }
    }
    for (int q = 0; q < b.nv; ++q) {
      const SvdPiece pc = pieces[b.v0 + q];
      const int64_t n = (int64_t)k * pc.cols;
      for (int64_t e = tid; e < n; e += kSvdThreads) {
        const int j = (int)(e / pc.cols);
        const int64_t c = pc.c0 + (e - (int64_t)j * pc.cols);
        Vt[pc.off + e] = V[c + (int64_t)pm[j] * C] * (absorb == 2 ? Ss[j] : sg * vs);
      }
    }
    return;
  }
  if (Sk)
    for (int j = tid; j < k; j += kSvdThreads) Sk[b.ks + j] = Ss[j] / vs;
  for (int q = 0; q < b.nu; ++q) {
    const SvdPiece pc = pieces[b.u0 + q];
    const int64_t n = (int64_t)pc.rows * k;
    for (int64_t e = tid; e < n; e += kSvdThreads) {
      const int i = (int)(e / k), j = (int)(e - (int64_t)i * k);
      const int64_t r = pc.r0 + i, pj = pm[j];
      const double s = Ss[j];
      double v;
      if (!b.trans) {
        const double w = W[r + pj * R];
        v = absorb == 1 ? w : (s > 0.0 ? vs * w / s : 0.0);
      } else {
        v = V[r + pj * C];
        v *= absorb == 1 ? s : vs;
      }
      U[pc.off + e] = v;
    }
  }
  for (int q = 0; q < b.nv; ++q) {
    const SvdPiece pc = pieces[b.v0 + q];
    const int64_t n = (int64_t)k * pc.cols;
    for (int64_t e = tid; e < n; e += kSvdThreads) {
      const int j = (int)(e / pc.cols);
      const int64_t c = pc.c0 + (e - (int64_t)j * pc.cols), pj = pm[j];
      const double s = Ss[j];
      double v;
      if (!b.trans) {
        v = V[c + pj * C];
        v *= absorb == 2 ? s : vs;
      } else {
        const double w = W[c + pj * R];
        v = absorb == 2 ? w : (s > 0.0 ? vs * w / s : 0.0);
      }
      Vt[pc.off + e] = v;
    }
  }
}

struct TupleEntry {
  int x;
  int64_t first, extent;
};
using TupleMap = std::unordered_map<std::vector<int>, TupleEntry, VecHash>;

int fused_label(int group, const std::vector<Leg>& legs, int l0, const std::vector<int>& pos) {
  if (group == SYM_SU2) return legs[l0].labels[pos[0]];  // rank 2: the spin of the one leg
  int k = 0;
  for (size_t i = 0; i < pos.size(); ++i) {
    const Leg& L = legs[l0 + i];
    k = group == SYM_Z2F ? (k ^ L.labels[pos[i]]) : k + L.dir * L.labels[pos[i]];
  }
  return k;
}

// Every label tuple of legs [l0, l1), lexicographic (first leg slowest),
// grouped by the block label x = partner(fused label), with its first
// row (column) inside the block.
TupleMap enumerate_tuples(int group, const std::vector<Leg>& legs, int l0, int l1, bool columns, int total,
                          std::unordered_map<int, int64_t>& extent) {
  TupleMap out;
  const int k = l1 - l0;
  std::vector<int> pos(k, 0);
  while (true) {
    const int f = fused_label(group, legs, l0, pos);
    const int x = !columns || group == SYM_SU2 ? f : group == SYM_Z2F ? (total ^ f) : total - f;
    int64_t e = 1;
    for (int i = 0; i < k; ++i) e *= legs[l0 + i].degens[pos[i]];
    int64_t& acc = extent[x];
    out[pos] = TupleEntry{x, acc, e};
    acc += e;
    int i = k - 1;
    while (i >= 0 && ++pos[i] == (int)legs[l0 + i].labels.size()) pos[i--] = 0;
    if (i < 0) break;
  }
  return out;
}

}  // namespace

struct SvdPlan {
  Tensor T;
  int nrow = 0;
  bool eig = false;  // eigendecomposition plan (sym_eig_plan)
  std::vector<int> xs;            // block labels, ascending
  std::vector<SvdBlock> blocks;   // ascending x
  std::vector<SvdPiece> tpieces;  // grouped by block
  TupleMap rows, cols;
  int64_t nsv = 0, work_elems = 0;
  int64_t smem32 = 0;      // dynamic shared memory of the Jacobi launch (FP32 sweeps by column blocks)
  std::vector<int> order;  // launch order: blocks by decreasing work
  bool dry = false;
  bool bonded = false;

  DeviceArena arena;
  SvdBlock* d_blocks = nullptr;
  double* work = nullptr;
  int* perm = nullptr;
  int* sweeps = nullptr;
  long long* rotations = nullptr;
  SvdPiece* d_pieces = nullptr;  // T pieces, then U and V pieces of the last bond
  size_t pieces_cap = 0;

  ~SvdPlan() {
    if (d_pieces) cudaFree(d_pieces);
  }

  void upload_blocks() {
    std::vector<SvdBlock> launch;
    for (int i : order) launch.push_back(blocks[i]);
    cudaError_t e = cudaMemcpy(d_blocks, launch.data(), launch.size() * sizeof(SvdBlock), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("svd plan upload: ") + cudaGetErrorString(e));
  }

  void upload_pieces(const std::vector<SvdPiece>& all) {
    cudaError_t e = cudaDeviceSynchronize();  // no launch of this plan may still read the old lists
    if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("svd plan upload: ") + cudaGetErrorString(e));
    if (all.size() > pieces_cap) {
      if (d_pieces) cudaFree(d_pieces);
      d_pieces = nullptr;
      pieces_cap = 0;
      e = cudaMalloc(&d_pieces, all.size() * sizeof(SvdPiece));
      if (e != cudaSuccess) {
        d_pieces = nullptr;
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? SYM_ERR_OOM : SYM_ERR_CUDA,
             std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
      }
      pieces_cap = all.size();
    }
    e = cudaMemcpy(d_pieces, all.data(), all.size() * sizeof(SvdPiece), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) fail(SYM_ERR_CUDA, std::string("svd plan upload: ") + cudaGetErrorString(e));
  }
};

std::unique_ptr<SvdPlan> plan_svd(const Tensor& T, int nrow, bool eig) {
  const char* what = eig ? "blockwise eigendecomposition" : "blockwise SVD";
  if (T.group == SYM_SU2U1) fail(SYM_ERR_UNSUPPORTED, std::string(what) + " of SU(2) x U(1) tensors is not built");
  if (T.group == SYM_SU2 && T.rank != 2)
    fail(SYM_ERR_UNSUPPORTED, std::string(what) + " of SU(2) tensors is built for rank 2 (the block-diagonal form)");
  if (T.rank < 2 || nrow < 1 || nrow >= T.rank) fail(SYM_ERR_ARG, "SVD needs rank >= 2 and 1 <= nrow < rank");
  if (eig) {  // a square matrix: the column legs are the row legs reversed, total label 0
    if (T.rank != 2 * nrow) fail(SYM_ERR_ARG, "eigendecomposition needs rank = 2 nrow");
    for (int l = 0; l < nrow; ++l)
      if (!T.legs[l].same_content(T.legs[nrow + l]) || T.legs[l].dir != -T.legs[nrow + l].dir)
        fail(SYM_ERR_INCOMPATIBLE_LEGS,
             "eigendecomposition: column leg " + std::to_string(nrow + l) + " must be row leg " + std::to_string(l) +
                 " reversed (same labels and degeneracies, opposite direction)");
    if (T.group != SYM_SU2 && T.total != 0) fail(SYM_ERR_ARG, "eigendecomposition needs total label 0");
  }
  auto P = std::make_unique<SvdPlan>();
  P->T = T;
  P->nrow = nrow;
  P->eig = eig;
  std::unordered_map<int, int64_t> mext, next;
  P->rows = enumerate_tuples(T.group, T.legs, 0, nrow, false, T.total, mext);
  P->cols = enumerate_tuples(T.group, T.legs, nrow, T.rank, true, T.total, next);
  for (auto& kv : mext)
    if (next.count(kv.first)) P->xs.push_back(kv.first);
  std::sort(P->xs.begin(), P->xs.end());
  if (P->xs.empty()) fail(SYM_ERR_ARG, "the tensor has no blocks");
  std::unordered_map<int, int> slot_of;
  for (int x : P->xs) {
    const int64_t m = mext[x], n = next[x];
    if (m >= (int64_t)1 << 31 || n >= (int64_t)1 << 31) fail(SYM_ERR_UNSUPPORTED, "SVD block too large");
    SvdBlock b{};
    b.m = (int)m;
    b.n = (int)n;
    b.trans = m < n;
    b.R = (int)std::max(m, n);
    b.C = (int)std::min(m, n);
    b.slot = (int)P->blocks.size();
    b.vscale = T.group == SYM_SU2 ? std::sqrt((double)x + 1.0) : 1.0;
    b.eig = eig ? 1 : 0;
    // SU(2) with an incoming row leg: the dense block is (-1)^{2j} M_x / sqrt(2j+1) (x) 1
    b.sgn = (eig && T.group == SYM_SU2 && T.legs[0].dir == -1 && (x & 1)) ? -1.0 : 1.0;
    if (eig && m != n) fail(SYM_ERR_ARG, "internal: eigendecomposition block is not square");
    // FP32 sweeps by column blocks when a block pair of W and V fits the
    // shared memory two CTAs of an SM can have, rows up to 12 per lane
    {
      const int bw = (b.C + kColBlocks - 1) / kColBlocks;
      const int64_t bytes = 2 * (int64_t)bw * (b.R + b.C + 1) * (int64_t)sizeof(float);
      const bool ok = b.C >= kColBlocks * 2 && b.R <= 32 * 12;
      b.bw = (ok && bytes <= kSvdSmem32Max) ? bw : 0;
      // FP64 by column blocks for the SVD only: on the shifted symmetric blocks of
      // the eigendecomposition that order took up to 6 FP64 sweeps where the
      // order by pairs takes 4 (two-site density matrix: 29.8 against 29.0 ms;
      // two-site SVD: 20.4 against 22.3 ms)
      b.bw64 = (ok && !eig && 2 * bytes <= kSvdSmem32Max) ? bw : 0;
      if (b.bw) P->smem32 = std::max<int64_t>(P->smem32, b.bw64 ? 2 * bytes : bytes);
    }
    b.w = P->work_elems;
    b.s = P->nsv;
    // W, V, norms, sorted S, A, the Newton-Schulz factor (doubles), W and V in FP32
    const int64_t rc = (int64_t)b.R * b.C, cc = (int64_t)b.C * b.C;
    P->work_elems += 2 * rc + 2 * cc + 2 * (int64_t)b.C + (rc + cc + 1) / 2 + 1;
    P->nsv += b.C;
    slot_of[x] = b.slot;
    P->blocks.push_back(b);
  }
  // tensor blocks, grouped by diagonal block
  std::vector<std::vector<SvdPiece>> per(P->blocks.size());
  for (int64_t s = 0; s < T.nsec(); ++s) {
    std::vector<int> rt(T.pos.begin() + s * T.rank, T.pos.begin() + s * T.rank + nrow);
    std::vector<int> ct(T.pos.begin() + s * T.rank + nrow, T.pos.begin() + (s + 1) * T.rank);
    const TupleEntry& r = P->rows.at(rt);
    const TupleEntry& c = P->cols.at(ct);
    if (r.x != c.x) fail(SYM_ERR_ARG, "internal: block outside the diagonal");
    const SvdBlock& b = P->blocks[slot_of.at(r.x)];
    if (r.first + r.extent > b.m || c.first + c.extent > b.n || r.extent * c.extent != T.block_size(s))
      fail(SYM_ERR_ARG, "internal: block outside its matrix");
    per[b.slot].push_back(SvdPiece{T.offs[s], (int)r.first, (int)c.first, (int)r.extent, (int)c.extent});
  }
  for (auto& b : P->blocks) {
    b.t0 = (int)P->tpieces.size();
    b.nt = (int)per[b.slot].size();
    P->tpieces.insert(P->tpieces.end(), per[b.slot].begin(), per[b.slot].end());
  }
  for (size_t i = 0; i < P->blocks.size(); ++i) P->order.push_back((int)i);
  std::stable_sort(P->order.begin(), P->order.end(), [&](int a, int c) {
    const SvdBlock &A = P->blocks[a], &B = P->blocks[c];
    return (double)A.R * A.C * A.C > (double)B.R * B.C * B.C;
  });
  const char* dry = std::getenv("SYM_PLAN_DRYRUN");
  P->dry = dry && dry[0] == '1';
  if (!P->dry) {
    P->d_blocks = static_cast<SvdBlock*>(P->arena.alloc(P->blocks.size() * sizeof(SvdBlock), false));
    P->work = static_cast<double*>(P->arena.alloc(P->work_elems * sizeof(double), true));
    P->perm = static_cast<int*>(P->arena.alloc(P->nsv * sizeof(int), true));
    P->sweeps = static_cast<int*>(P->arena.alloc(2 * P->blocks.size() * sizeof(int), true));
    P->rotations = static_cast<long long*>(P->arena.alloc(2 * P->blocks.size() * sizeof(long long), true));
    P->upload_blocks();
    P->upload_pieces(P->tpieces);
  }
  return P;
}

}  // namespace sym

struct sym_svd_s {
  std::unique_ptr<sym::SvdPlan> p;
};

namespace {

void need(bool ok, const char* msg) {
  if (!ok) sym::fail(SYM_ERR_ARG, msg);
}

void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) sym::fail(SYM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

int sym_svd_plan(sym_tensor T, int nrow, sym_svd* out, int* nblocks, int64_t* nsv) {
  return sym::guard([&] {
    need(T != nullptr && out != nullptr, "T or out is NULL");
    auto P = sym::plan_svd(T->t, nrow, false);
    if (nblocks) *nblocks = (int)P->blocks.size();
    if (nsv) *nsv = P->nsv;
    *out = new sym_svd_s{std::move(P)};
    return SYM_OK;
  });
}

int sym_eig_plan(sym_tensor T, int nrow, sym_svd* out, int* nblocks, int64_t* nev) {
  return sym::guard([&] {
    need(T != nullptr && out != nullptr, "T or out is NULL");
    auto P = sym::plan_svd(T->t, nrow, true);
    if (nblocks) *nblocks = (int)P->blocks.size();
    if (nev) *nev = P->nsv;
    *out = new sym_svd_s{std::move(P)};
    return SYM_OK;
  });
}

int sym_svd_blocks(sym_svd plan, int* x, int* m, int* n) {
  return sym::guard([&] {
    need(plan != nullptr, "plan is NULL");
    const auto& P = *plan->p;
    for (size_t i = 0; i < P.blocks.size(); ++i) {
      if (x) x[i] = P.xs[i];
      if (m) m[i] = P.blocks[i].m;
      if (n) n[i] = P.blocks[i].n;
    }
    return SYM_OK;
  });
}

namespace {
void launch_jacobi(sym::SvdPlan& P, const double* T, double* S, void* stream) {
  if (P.dry) sym::fail(SYM_ERR_UNSUPPORTED, "plan was built with SYM_PLAN_DRYRUN=1 and cannot run");
  static int attr_set = -1;  // dynamic shared memory the kernel is allowed (set once to the maximum)
  if (attr_set < 0) {
    cudaError_t e = cudaFuncSetAttribute(sym::svd_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sym::kSvdSmem32Max);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(sym::svd_jacobi_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) sym::fail(SYM_ERR_CUDA, std::string("svd_jacobi_kernel attribute: ") + cudaGetErrorString(e));
    attr_set = 1;
  }
  sym::svd_jacobi_kernel<<<(unsigned)P.blocks.size() * sym::kSvdCluster, sym::kSvdThreads, (size_t)P.smem32,
                           static_cast<cudaStream_t>(stream)>>>(
      P.d_blocks, P.d_pieces, T, P.work, S, P.perm, P.sweeps, P.rotations, sym::device_error_word());
  check_launch("svd_jacobi_kernel");
}
}  // namespace

int sym_eig_execute(sym_svd plan, const double* T, double* lambda, void* stream) {
  return sym::guard([&] {
    need(plan != nullptr && T != nullptr && lambda != nullptr, "plan, T or lambda is NULL");
    need(plan->p->eig, "not an eigendecomposition plan (sym_eig_plan)");
    launch_jacobi(*plan->p, T, lambda, stream);
    return SYM_OK;
  });
}

int sym_svd_execute(sym_svd plan, const double* T, double* S, void* stream) {
  return sym::guard([&] {
    need(plan != nullptr && T != nullptr && S != nullptr, "plan, T or S is NULL");
    auto& P = *plan->p;
    need(!P.eig, "an eigendecomposition plan runs with sym_eig_execute");
    launch_jacobi(P, T, S, stream);
    return SYM_OK;
  });
}

int sym_svd_stats(sym_svd plan, int fp32, int* sweeps, int64_t* rotations) {
  return sym::guard([&] {
    need(plan != nullptr, "plan is NULL");
    need(fp32 == 0 || fp32 == 1, "fp32 must be 0 (the FP64 sweeps) or 1 (the FP32 sweeps)");
    auto& P = *plan->p;
    if (P.dry) sym::fail(SYM_ERR_UNSUPPORTED, "plan was built with SYM_PLAN_DRYRUN=1 and cannot run");
    const size_t nb = P.blocks.size();
    std::vector<int> sw(2 * nb);
    std::vector<long long> r(2 * nb);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(sw.data(), P.sweeps, sw.size() * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r.data(), P.rotations, r.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) sym::fail(SYM_ERR_CUDA, std::string("svd stats: ") + cudaGetErrorString(e));
    const int k = fp32;
    for (size_t i = 0; i < nb; ++i) {
      if (sweeps) sweeps[i] = sw[2 * i + k];
      if (rotations) rotations[i] = r[2 * i + k];
    }
    return SYM_OK;
  });
}

int sym_svd_bond(sym_svd plan, const int* keep, sym_tensor* U, sym_tensor* V) {
  return sym::guard([&] {
    need(plan != nullptr && keep != nullptr && U != nullptr && V != nullptr, "plan, keep, U or V is NULL");
    auto& P = *plan->p;
    const sym::Tensor& T = P.T;
    sym::Leg bu, bv;
    bu.dir = -1;
    bv.dir = 1;
    for (size_t i = 0; i < P.blocks.size(); ++i) {
      need(keep[i] >= 0 && keep[i] <= P.blocks[i].C, "keep[b] must be in 0..min(m, n) of block b");
      if (keep[i] > 0) {
        bu.labels.push_back(P.xs[i]);
        bu.degens.push_back(keep[i]);
      }
    }
    need(!bu.labels.empty(), "at least one singular vector must be kept");
    bv.labels = bu.labels;
    bv.degens = bu.degens;
    std::vector<sym::Leg> lu(T.legs.begin(), T.legs.begin() + P.nrow), lv{bv};
    lu.push_back(bu);
    lv.insert(lv.end(), T.legs.begin() + P.nrow, T.legs.end());
    const sym::Tree tr = T.group == SYM_SU2 ? sym::Tree::comb(2) : sym::Tree{};
    sym::Tensor tu = sym::make_tensor(T.group, lu, 0, tr);
    sym::Tensor tv = sym::make_tensor(T.group, lv, T.total, tr);
    std::unordered_map<int, int> slot_of;
    for (size_t i = 0; i < P.xs.size(); ++i) slot_of[P.xs[i]] = (int)i;
    std::vector<std::vector<sym::SvdPiece>> pu(P.blocks.size()), pv(P.blocks.size());
    for (int64_t s = 0; s < tu.nsec(); ++s) {
      std::vector<int> rt(tu.pos.begin() + s * tu.rank, tu.pos.begin() + s * tu.rank + P.nrow);
      const int x = tu.label(s, P.nrow);
      const auto& r = P.rows.at(rt);
      need(r.x == x, "internal: U block outside the diagonal");
      const int b = slot_of.at(x);
      pu[b].push_back(sym::SvdPiece{tu.offs[s], (int)r.first, 0, (int)r.extent, keep[b]});
    }
    for (int64_t s = 0; s < tv.nsec(); ++s) {
      std::vector<int> ct(tv.pos.begin() + s * tv.rank + 1, tv.pos.begin() + (s + 1) * tv.rank);
      const int x = tv.label(s, 0);
      const auto& c = P.cols.at(ct);
      need(c.x == x, "internal: V block outside the diagonal");
      const int b = slot_of.at(x);
      pv[b].push_back(sym::SvdPiece{tv.offs[s], 0, (int)c.first, keep[b], (int)c.extent});
    }
    std::vector<sym::SvdPiece> all(P.tpieces);
    int ks = 0;
    for (size_t b = 0; b < P.blocks.size(); ++b) {
      auto& B = P.blocks[b];
      B.keep = keep[b];
      B.ks = ks;
      ks += keep[b];
      B.u0 = (int)all.size();
      B.nu = (int)pu[b].size();
      all.insert(all.end(), pu[b].begin(), pu[b].end());
      B.v0 = (int)all.size();
      B.nv = (int)pv[b].size();
      all.insert(all.end(), pv[b].begin(), pv[b].end());
    }
    if (!P.dry) {
      P.upload_pieces(all);
      P.upload_blocks();
    }
    P.bonded = true;
    *U = new sym_tensor_s{std::move(tu)};
    *V = new sym_tensor_s{std::move(tv)};
    return SYM_OK;
  });
}

int sym_svd_factors(sym_svd plan, int absorb, double* U, double* V, double* Sk, void* stream) {
  return sym::guard([&] {
    need(plan != nullptr && U != nullptr && V != nullptr, "plan, U or V is NULL");
    need(absorb >= 0 && absorb <= 2, "absorb must be 0, 1 or 2");
    auto& P = *plan->p;
    if (P.dry) sym::fail(SYM_ERR_UNSUPPORTED, "plan was built with SYM_PLAN_DRYRUN=1 and cannot run");
    if (!P.bonded) sym::fail(SYM_ERR_ARG, "sym_svd_bond must be called before sym_svd_factors");
    sym::svd_factor_kernel<<<(unsigned)P.blocks.size(), sym::kSvdThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        P.d_blocks, P.d_pieces, P.work, P.perm, U, V, Sk, absorb);
    check_launch("svd_factor_kernel");
    return SYM_OK;
  });
}

namespace {
// keep[b] from the values' magnitudes (SVD: the singular values; eig: |lambda|)
void truncate_values(const sym::SvdPlan& P, const double* S, int64_t chi, double cutoff, int* keep) {
  need(cutoff >= 0.0, "cutoff must be >= 0");
  struct Val {
    double v;
    int b, i;
  };
  std::vector<Val> vals;
  vals.reserve(P.nsv);
  for (size_t b = 0; b < P.blocks.size(); ++b)
    for (int i = 0; i < P.blocks[b].C; ++i) {
      const double s = S[P.blocks[b].s + i];
      const double v = P.eig ? std::fabs(s) : s;
      if (!(v >= 0.0) || !std::isfinite(v))
        sym::fail(SYM_ERR_NUMERIC, P.eig ? "eigenvalues must be finite" : "singular values must be finite and >= 0");
      vals.push_back(Val{v, (int)b, i});
    }
  // descending; ties: smaller x first, then the block's own order
  std::sort(vals.begin(), vals.end(), [](const Val& a, const Val& c) {
    if (a.v != c.v) return a.v > c.v;
    return a.b != c.b ? a.b < c.b : a.i < c.i;
  });
  const double vmax = vals.empty() ? 0.0 : vals[0].v;
  for (size_t b = 0; b < P.blocks.size(); ++b) keep[b] = 0;
  int64_t n = 0;
  for (const Val& x : vals) {
    const int w = P.T.group == SYM_SU2 ? P.xs[x.b] + 1 : 1;  // dense values one value stands for
    if (chi >= 0 && n + w > chi) break;
    if (cutoff > 0.0 && x.v <= cutoff * vmax) break;
    ++keep[x.b];
    n += w;
  }
}
}  // namespace

int sym_svd_truncation(sym_svd plan, const double* S, int64_t chi, double cutoff, int* keep) {
  return sym::guard([&] {
    need(plan != nullptr && S != nullptr && keep != nullptr, "plan, S or keep is NULL");
    need(!plan->p->eig, "an eigendecomposition plan truncates with sym_eig_truncation");
    truncate_values(*plan->p, S, chi, cutoff, keep);
    return SYM_OK;
  });
}

int sym_eig_truncation(sym_svd plan, const double* lambda, int64_t chi, double cutoff, int* keep) {
  return sym::guard([&] {
    need(plan != nullptr && lambda != nullptr && keep != nullptr, "plan, lambda or keep is NULL");
    need(plan->p->eig, "not an eigendecomposition plan (sym_eig_plan)");
    truncate_values(*plan->p, lambda, chi, cutoff, keep);
    return SYM_OK;
  });
}

int sym_svd_destroy(sym_svd plan) {
  delete plan;
  return SYM_OK;
}

}  // extern "C"
