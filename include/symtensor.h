/*
 * symtensor.h -- C ABI of the GB300 symmetric block-sparse contraction library.
 *
 * A symmetric tensor (S. Singh, arXiv:1203.2222) is stored as its degeneracy
 * blocks only.  This library builds the integer sector tables of such tensors
 * on the host and moves, recouples and multiplies the blocks on one GPU.
 *
 * Data model (Ch. 5 "Tensors as linear maps", Ch. 6 "Tree decompositions"):
 *   - A leg is a list of n labels with degeneracies and a direction
 *     (+1 'out', -1 'in').  U(1): labels are integer charges.  SU(2): labels
 *     are doubled spins 2j.  Fermion parity: 0 or 1.  SU(2) x U(1):
 *     64 q + 2j (see sym_tensor_create).  Labels are strictly increasing.
 *   - U(1): a block (sector) is one charge per leg with
 *       sum_out q - sum_in q == total   (charge conservation).
 *   - SU(2): the tensor is a tree decomposition; a sector is one spin per leg
 *     plus one spin per non-root node of the fusion tree, every node obeying
 *     the fusion rule |ja-jb| <= jc <= ja+jb (Ch. 5, Eq. fusionrules) and the
 *     root carrying spin 0 (the vector v of Ch. 6 is invariant).  Incoming
 *     legs carry a cup (Ch. 6); reversal of a leg is metadata only.
 *   - A tree over k legs is given as k-1 nodes (left, right): ids 0..k-1 are
 *     legs, node n has id k+n, the last node is the root and every node joins
 *     two adjacent leg ranges, left first.  NULL means the left comb
 *     ((0,1),2),...
 *   - Sectors are ordered lexicographically by leg label positions (leg 0
 *     slowest), then by node spins in node order.  Each block is a dense
 *     d_1 x ... x d_k array, row-major (last leg fastest); blocks are
 *     concatenated in sector order.  Block data lives in caller-owned device
 *     buffers of numel elements (float for SYM_PREC_BF16X3 plans, double for
 *     SYM_PREC_FP64 plans); the library never frees them.
 *
 * Handles (sym_tensor, sym_plan) are owned by the caller and freed with the
 * matching destroy call.  A sym_tensor holds structure only (host tables).
 * A sym_plan holds the precomputed tables of one operation (uploaded to the
 * device) and its scratch operand buffers; it is the precomputation of
 * symmetry-only data the thesis recommends reusing across iterations
 * (Ch. 6, "Discussion on computational performance").
 *
 * Environment: SYM_PLAN_DRYRUN=1 makes the *_plan calls build and
 * bounds-check their work lists on the host without touching the GPU; such
 * plans report statistics but refuse to execute (SYM_ERR_UNSUPPORTED).
 *
 * Errors: every call returns SYM_OK (0) or a negative SYM_ERR_* code;
 * sym_last_error() returns a thread-local message for the last failure.
 * Execution calls are asynchronous on the given CUDA stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream); they return SYM_ERR_CUDA if
 * a launch fails.  Device-side bounded waits that expire set a device error
 * word that sym_device_status() reports as SYM_ERR_TIMEOUT (SYM_ERR_NUMERIC
 * for an SVD block that did not converge).
 */
#ifndef SYMTENSOR_H
#define SYMTENSOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYM_OK 0
#define SYM_ERR_ARG (-1)               /* malformed argument */
#define SYM_ERR_INCOMPATIBLE_LEGS (-2) /* contracted legs differ or share a direction */
#define SYM_ERR_CUDA (-4)              /* a CUDA call failed */
#define SYM_ERR_TIMEOUT (-5)           /* a device-side bounded wait expired */
#define SYM_ERR_OOM (-6)               /* host or device allocation failed */
#define SYM_ERR_UNSUPPORTED (-7)       /* valid request outside what is built */
#define SYM_ERR_NUMERIC (-8)           /* an iterative method did not converge */

#define SYM_U1 1
#define SYM_SU2 2
#define SYM_Z2F 3 /* fermion parity: labels 0/1, fusion mod 2, swap of two odd charges -1 */
#define SYM_SU2U1 4 /* SU(2) x U(1): label = 64 q + 2j (0 <= 2j < 64), see sym_tensor_create */

/* Precision of a plan (the storage dtype follows from it). */
#define SYM_PREC_FP64 1   /* double blocks, FP64 gathers and FP64 GEMM (CUDA cores) */
#define SYM_PREC_BF16X3 2 /* float blocks, split-BF16 x3 tcgen05 GEMM, FP32 accumulate */

typedef struct {
  int n;              /* number of labels */
  const int* labels;  /* U(1) charges or SU(2) doubled spins, strictly increasing */
  const int* degens;  /* degeneracy d of every label, >= 1 */
  int dir;            /* +1 out, -1 in */
} sym_leg;

typedef struct sym_tensor_s* sym_tensor;
typedef struct sym_plan_s* sym_plan;

/* Last error message of the calling thread ("" if none). */
const char* sym_last_error(void);

/* Library build information, e.g. "symtensor sm_103a". */
const char* sym_version(void);

/* ---------------------------------------------------------------- tensors ---
 * sym_tensor_create: build the sector table of a tensor (host only, no GPU).
 *   group: SYM_U1, SYM_SU2 or SYM_Z2F (fermion parity of the thesis's
 *   conclusion: labels p = 0, 1 fuse by addition mod 2, the recoupling
 *   coefficients are 1, and exchanging two legs of odd parity multiplies a
 *   block by -1; total = 0 or 1; every permutation, fuse and contraction
 *   applies these swap signs, and nothing else differs from U(1)), or
 *   SYM_SU2U1 (the composite symmetry of the thesis's conclusion, the two
 *   groups acting component by component: a label is the pair (q, 2j)
 *   stored as 64 q + 2j with 0 <= 2j < 64, so that increasing labels sort by
 *   charge, then spin; a sector is a tree decomposition as for SU(2) on the
 *   spins whose charges obey the U(1) rule sum_out q - sum_in q = total; the
 *   recoupling coefficients and cups are the spins' alone; a fused label
 *   adds the charges and couples the spins).  0 <= rank <= 6 (rank 0 is a scalar).
 *   total: U(1) total charge Q (also for SYM_SU2U1); ignored for SU(2) (total spin is 0).
 *   tree: SU(2) and SU(2) x U(1) fusion tree as 2*(rank-1) ints, NULL = left comb; ignored otherwise.
 *   legs: rank leg descriptors (copied).
 * Errors: SYM_ERR_ARG for malformed legs or trees.                          */
int sym_tensor_create(int group, int rank, const sym_leg* legs, int total,
                      const int* tree, sym_tensor* out);
int sym_tensor_destroy(sym_tensor t);

/* group, rank, numel (elements of all blocks), nsec (number of sectors). */
int sym_tensor_info(sym_tensor t, int* group, int* rank, int64_t* numel,
                    int64_t* nsec);
/* Copy leg `leg` (labels/degens may be NULL to query *n first). */
int sym_tensor_leg(sym_tensor t, int leg, int* n, int* labels, int* degens,
                   int* dir);
/* Copy the tree (2*(rank-1) ints) of an SU(2) tensor. */
int sym_tensor_tree(sym_tensor t, int* nodes);
/* Sector table: labels receives nsec*(rank + max(rank-2,0)) ints (leg label
 * positions, then SU(2) non-root node spins 2j); offsets receives nsec+1
 * block offsets (exclusive prefix sum of block sizes).  Either may be NULL. */
int sym_tensor_sectors(sym_tensor t, int* labels, int64_t* offsets);

/* ------------------------------------------------------------- operations ---
 * Each operation is planned once on the host (structure only; the result's
 * structure handle is returned) and executed any number of times on device
 * data.  `precision` selects the data type the plan works in.
 *
 * sym_permute_plan: PERMUTE of Ch. 6 -- output leg n is input leg perm[n];
 *   SU(2) output tree tree_out (NULL = left comb), the blocks recoupled by
 *   v' = Gamma(tau, p, tau') v with 6j recoupling and swap factors.
 * sym_fuse_plan: FUSE of Ch. 6 -- legs first and first+1 (equal directions)
 *   become one leg (fused labels ascending; within a fused label the pairs
 *   (la, lb) are ordered with la slowest and (t_a, t_b) row-major).  For
 *   SU(2) the input is first taken to the tree where the two legs share a
 *   node (NEWTREE), the output tree is the left comb.
 * sym_fuse_n_plan: legs first..first+nlegs-1 (nlegs >= 2, equal directions)
 *   become one leg, fused pairwise from the left: ((l_f, l_f+1), l_f+2), ...
 *   (the fused leg's labels and order are those of nlegs-1 sym_fuse_plan
 *   steps).  For nlegs > 2 the plan runs the pairwise steps in order through
 *   two device scratch buffers it allocates and owns (the largest
 *   intermediate); its launches are not recorded by sym_plan_profile.
 * sym_split_plan: SPLIT of Ch. 6 -- leg `leg` is split into the two legs
 *   parts[0], parts[1], which must fuse exactly to it; SU(2) output tree is
 *   the left comb.
 * sym_plan_execute: run a permute/fuse/split plan: out = op(in).          */
int sym_permute_plan(sym_tensor in, const int* perm, const int* tree_out,
                     int precision, sym_tensor* out, sym_plan* plan);
int sym_fuse_plan(sym_tensor in, int first, int precision, sym_tensor* out,
                  sym_plan* plan);
int sym_fuse_n_plan(sym_tensor in, int first, int nlegs, int precision,
                    sym_tensor* out, sym_plan* plan);
int sym_split_plan(sym_tensor in, int leg, const sym_leg* parts, int precision,
                   sym_tensor* out, sym_plan* plan);
int sym_plan_execute(sym_plan plan, const void* in, void* out, void* stream);

/* sym_contract_plan: the five-step contraction of Ch. 5 ("Multiplication of
 *   two tensors", Eq. multi1-multi5) and Ch. 6 ("Multiplication of two
 *   tensors"): legs pairsA[i] of A and pairsB[i] of B are summed over; each
 *   pair must have identical labels/degeneracies and opposite directions
 *   (SYM_ERR_INCOMPATIBLE_LEGS otherwise).  The result C has A's free legs
 *   (in order) then B's free legs; U(1) total charge QA + QB; SU(2) tree
 *   tree_c, NULL = comb over A's free legs and comb over B's free legs joined
 *   at the root.  Steps on the device: gather A and B into per-sector matrix
 *   form (block transpose; SU(2): recoupling by precomputed 6j/swap
 *   coefficients), one grouped per-sector GEMM (blockwise product,
 *   Ch. 5 Eq. blockmult), scatter into C's blocks.  U(1) sectors whose
 *   matrix of B is at most 4 x 4 (an MPO or physical leg on the contracted
 *   side) skip the matrix form: their product is taken directly on A's and
 *   C's blocks with B's sector matrix as coefficients (one streaming pass;
 *   the gradient of B is an atomic reduction into dB).
 * sym_contract: C = contract(A, B) on device buffers.
 * sym_contract_backward: dA, dB = gradient of <dC, C> with respect to A's
 *   and B's blocks (adjoint on the same sector tables); dA or dB may be NULL
 *   to skip it.  Buffers are overwritten, not accumulated.
 *   sym_contract_backward reads the tensor-core operand forms of A and B
 *   that the plan's last sym_contract gathered when that call received the
 *   same A and B pointers (A and B must then not have been modified in
 *   between, as for any saved autograd input); otherwise it gathers them
 *   again from A and B.
 *   Both are asynchronous on `stream`.  The GEMM launches of one call run
 *   concurrently on side streams that the plan creates on first use, forked
 *   from `stream` and joined back into it with events (in a stream capture
 *   they become graph dependencies).  A plan owns its scratch buffers:
 *   executions of one plan must not overlap (serialize calls that share a
 *   plan across streams or threads).
 * sym_plan_stats: useful flops of one forward (sum over sectors of 2 m n k),
 *   and bytes of A, B and C blocks in the plan's data type.              */
int sym_contract_plan(sym_tensor A, sym_tensor B, int npairs, const int* pairsA,
                      const int* pairsB, const int* tree_c, int precision,
                      sym_tensor* C, sym_plan* plan);
int sym_contract(sym_plan plan, const void* A, const void* B, void* C,
                 void* stream);
int sym_contract_backward(sym_plan plan, const void* A, const void* B,
                          const void* dC, void* dA, void* dB, void* stream);
/* sym_contract_batch_plan: nprob independent contractions of the same kind
 *   (the contraction of Ch. 5, "Multiplication of two tensors", for every
 *   pair A[i], B[i] over the same leg pairs) as ONE plan: their blocks live in
 *   packed buffers, problem i's A at element offsets[i] of the packed A, its
 *   B at offsets[nprob + 1 + i] of the packed B and its C at
 *   offsets[2 (nprob + 1) + i] of the packed C (offsets: 3 (nprob + 1)
 *   int64, written; each list ends with the packed size).  C[i] (nprob
 *   handles, written, owned by the caller) are the result structures, as
 *   sym_contract_plan makes them.  sym_contract / sym_contract_backward on
 *   the packed buffers then run every phase of all problems in one launch per
 *   kernel (GEMM tiles of all problems scheduled longest reduction first).
 *   The thesis runs its contractions one at a time; grouping is this
 *   library's.  Problems are planned in parallel on the host.  Errors as
 *   sym_contract_plan (the first failing problem's).                     */
int sym_contract_batch_plan(int nprob, const sym_tensor* A, const sym_tensor* B,
                            int npairs, const int* pairsA, const int* pairsB,
                            int precision, sym_tensor* C, int64_t* offsets,
                            sym_plan* plan);
int sym_plan_stats(sym_plan plan, double* flops_fwd, int64_t* bytes_a,
                   int64_t* bytes_b, int64_t* bytes_c);
int sym_plan_destroy(sym_plan plan);

/* GEMM sectors of a contraction plan (forward, dA and dB GEMMs of every
 * sector): *nsec receives their number and mnk (may be NULL) 4*nsec ints
 * (m, n, k, kernel) with kernel 0 = tcgen05 split-BF16, 1 = CUDA cores. */
int sym_plan_gemm_shapes(sym_plan plan, int* nsec, int* mnk);

/* Per-phase device timing of a plan's own launches.  sym_plan_profile(p, 1)
 * clears and starts recording a CUDA event pair around every launch (on the
 * launch stream); 0 stops.  sym_plan_profile_read synchronizes on the
 * recorded events and returns, for one phase, the number of launches, their
 * summed device time, and their algorithmic bytes (block data read once +
 * destination written once) and useful flops (sum of 2 m n k).           */
#define SYM_PHASE_FWD_GATHER 0
#define SYM_PHASE_FWD_GEMM 1 /* forward sectors on the tcgen05 GEMM */
#define SYM_PHASE_FWD_SCATTER 2
#define SYM_PHASE_BWD_GATHER 3
#define SYM_PHASE_BWD_GEMM 4
#define SYM_PHASE_BWD_SCATTER 5
#define SYM_PHASE_TRANSFORM 6
#define SYM_PHASE_FWD_GEMM_CUDA_CORES 7 /* forward sectors on the CUDA-core GEMMs */
#define SYM_PHASE_BWD_GEMM_CUDA_CORES 8
#define SYM_PHASE_FWD_DIRECT 9  /* forward sectors contracted directly on the blocks */
#define SYM_PHASE_BWD_DIRECT 10 /* their dA and dB */
int sym_plan_profile(sym_plan plan, int enable);
int sym_plan_profile_read(sym_plan plan, int phase, int* launches,
                          double* total_ms, double* bytes, double* flops);

/* The same records by kernel: sym_plan_profile_kernel returns launches,
 * summed device time, algorithmic bytes and useful flops of the recorded
 * launches of one kernel (SYM_KERNEL_*), over all phases.                */
#define SYM_KERNEL_BOX 0       /* block movement, general form (tiles, recoupling sums) */
#define SYM_KERNEL_BOX_FLAT 1  /* block movement, launches of flat linear items only */
#define SYM_KERNEL_GEMM_TC 2   /* tcgen05 split-BF16 x3 grouped GEMM */
#define SYM_KERNEL_GEMM_TILE 3 /* CUDA cores, 64 x 64 tiles */
#define SYM_KERNEL_GEMM_WIDE 4 /* CUDA cores, 256 x 16 tiles */
#define SYM_KERNEL_GEMM_THIN 5 /* CUDA cores, m, n <= 8, split reduction */
#define SYM_KERNEL_GEMM_ROWS 6 /* CUDA cores, k, n <= 16 */
#define SYM_KERNEL_DIRECT 7    /* sectors with a tiny matrix, contracted on the blocks */
#define SYM_KERNEL_COUNT 8
int sym_plan_profile_kernel(sym_plan plan, int kernel, int* launches,
                            double* total_ms, double* bytes, double* flops);

/* Planning parameters: the kernel choice per GEMM shape and the schedule of
 * the grouped launches.  Every plan built after sym_tune_set uses them (plans
 * already built keep theirs); sym_tune_epoch counts the sym_tune_set calls,
 * so a caller that caches plans can tell when to rebuild them.  Defaults
 * (SYM_TC_MIN_MN, SYM_TC_MIN_K, SYM_TC_MAX_K and SYM_DIRECT_MAX in the
 * environment override the first four at load):
 *   tc_min_mn 64, tc_min_k 48, tc_max_k 16384: a GEMM (m x n, reduction k)
 *     runs on the tensor cores when m, n >= tc_min_mn and tc_min_k <= k <=
 *     tc_max_k (and m, n > 8, not k, n <= 16), else on the CUDA cores;
 *   direct_max 4 (0..4): U(1) sectors whose B matrix is at most direct_max
 *     square are contracted directly on the blocks;
 *   direct_chunk 1024 (multiple of 32): positions per direct work item;
 *   rows_spans 8 (1..64): rows kernel, row runs per warp tile;
 *   splitk_ctas 2 (0..64): CUDA-core tile GEMMs split their reductions until
 *     a launch has splitk_ctas CTAs per SM (0: never split);
 *   thin_slice 4096 (multiple of 256): thin GEMMs, reduction per CTA;
 *   tc_order 0: tcgen05 tiles longest reduction first; 1: in sector order;
 *   tc_group 8 (0..256): inside a sector the tcgen05 tiles run in groups of
 *     tc_group row tiles, all column tiles of a group before the next
 *     group, so that a wave of CTAs shares its operand panels in L2 (0: row
 *     by row);
 *   direct_mixed 1: a contraction may mix direct sectors with GEMM sectors;
 *     0: its sectors go direct only when all of them qualify (no extra
 *     launches for a few tiny sectors of a large contraction);
 *   tc_all 0: 1 sends every GEMM of a split-BF16 plan with k <= tc_max_k to
 *     the tensor cores (small sectors padded into 128 x 128 tiles), so a
 *     GEMM phase is one launch instead of one per CUDA-core kind; longer
 *     reductions keep the CUDA-core kernels, which split them across CTAs.
 * sym_tune_set rejects a value out of range with SYM_ERR_ARG.             */
typedef struct {
  int tc_min_mn, tc_min_k, tc_max_k;
  int direct_max, direct_chunk;
  int rows_spans, splitk_ctas, thin_slice, tc_order, tc_group;
  int direct_mixed, tc_all;
} sym_tune;
int sym_tune_get(sym_tune* out);
int sym_tune_set(const sym_tune* in);
int sym_tune_epoch(int* epoch);

/* Number of kernel launches the last execution call on this plan issued. */
int sym_plan_launches(sym_plan plan, int* launches);

/* ------------------------------------------------ SU(2) recoupling (host) ---
 * The symmetry-only data the planner precomputes, exposed for inspection;
 * no GPU is touched.  Spins are doubled.
 * sym_su2_F: the recoupling coefficient F^{jd je}_{ja jb jc J} of Ch. 5,
 *   Eq. fmove, evaluated from the Wigner 6j symbol (Eq. sixj, Racah's
 *   formula): the overlap <(a,b)d, c; J | a, (b,c)e; J>; 0 if not allowed.
 * sym_su2_gamma: the matrix Gamma(tau, p, tau') of Ch. 6 (Eq. permsu2) for
 *   fixed leg spins: out[o * n_in + i] = < tau'; labelling o | p(tau; labelling i) >,
 *   where output leg n is input leg perm[n] and labellings enumerate the
 *   non-root node spins of each tree in sector order.  Pass G = NULL to
 *   query n_in / n_out; labels_in / labels_out (may be NULL) receive the
 *   labellings, max(rank-2,0) ints each.  Trees as in sym_tensor_create.   */
int sym_su2_F(int jd, int je, int ja, int jb, int jc, int J, double* out);
int sym_su2_gamma(int rank, const int* spins, const int* tree_in, const int* perm,
                  const int* tree_out, int* n_in, int* n_out, double* G,
                  int* labels_in, int* labels_out);

/* ------------------------------------------ contraction without allocation ---
 * sym_contract_noalloc: C = contract(A, B) exactly as sym_contract_plan +
 *   sym_contract with tree_c = NULL would compute it, for callers that cannot
 *   call cudaMalloc (code that must not enter the CUDA allocator, or that runs
 *   next to a framework owning all device memory).  It allocates no device
 *   memory: its work lists and operand scratch live in one file-scope
 *   __device__ array of 32 MiB that every GPU loading the library holds until
 *   exit.  The thesis has no counterpart; this is a deployment variant.
 *   A, B: structures; a, b: their device data; c: device buffer for the
 *   result, whose layout is that of the structure sym_contract_plan(A, B,
 *   npairs, pairsA, pairsB, NULL, precision, ...) returns (numel elements of
 *   double for SYM_PREC_FP64, float for SYM_PREC_BF16X3); caller-owned.
 *   Asynchronous on `stream`.  The first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) with that device current;
 *   make that first call before any stream capture.  Every call copies its
 *   work lists into the shared array, which keeps the last call's contents
 *   (nothing in it needs to start at zero: the call's own gathers and
 *   zero-fill items write everything its GEMMs read), so calls whose
 *   executions overlap on the GPU (other streams, other threads) race:
 *   serialize them.  Plans are cached on the host under the contents of A's
 *   and B's structures (legs, total, tree), the pairs, the precision and the
 *   sym_tune epoch, so a destroyed handle whose address is reused never
 *   reaches a stale plan and sym_tune_set takes effect on the next call; at
 *   most 64 plans are kept, the oldest dropped first.  A bounded device-side
 *   wait that expires sets a second static error word, which
 *   sym_device_status reads and clears with the library's own.  Errors:
 *   SYM_ERR_UNSUPPORTED (with the needed size) if the contraction needs more
 *   than 32 MiB of scratch, the argument errors of sym_contract_plan,
 *   SYM_ERR_CUDA if a copy or launch fails.                                  */
int sym_contract_noalloc(sym_tensor A, sym_tensor B, int npairs,
                         const int* pairsA, const int* pairsB, int precision,
                         const void* a, const void* b, void* c, void* stream);

/* Device error word: SYM_OK, SYM_ERR_TIMEOUT if a bounded wait in a
 * persistent kernel expired, or SYM_ERR_NUMERIC if an SVD block did not
 * converge, since the last call (the word is then cleared).  Synchronizes the
 * device. */
int sym_device_status(void);

/* Test of the failure detection (no counterpart in the thesis): runs, on the
 * legacy default stream, one bounded mbarrier wait of the kind the
 * tensor-core kernel's waits are, for a phase that nothing completes, and
 * synchronizes.  The wait expires after limit_us microseconds (1 ..
 * 2,000,000) and sets SYM_ERR_TIMEOUT in the library's device error word
 * (word = 0) or in sym_contract_noalloc's static one (word = 1), which the
 * next sym_device_status() then reports and clears; the context stays
 * usable.  Nothing faults and nothing waits without a limit.  Errors:
 * SYM_ERR_ARG for a limit or word out of range, SYM_ERR_CUDA if the launch
 * or the synchronization fails. */
int sym_wait_probe(int limit_us, int word);

/* ------------------------------------------ blockwise factorization (SVD) ---
 * Singular value decomposition of a symmetric tensor seen as a matrix
 * (Ch. 5, "Factorization of a matrix", Eq. svd0 and svd1; Ch. 6, "Matrix
 * multiplication and factorizations"): rows = legs 0..nrow-1, columns = the
 * other legs.  The matrix is block diagonal in the fused label x of its row
 * legs (U(1): sum of dir*q over the row legs; fermion parity: their parity
 * sum mod 2); block M_x is m_x x n_x, its rows the row-label tuples in
 * lexicographic order (leg 0 slowest, prod d rows each), its columns the
 * column-label tuples likewise, and every tensor block is the row-major
 * sub-matrix at its tuples' first row and column.  Every M_x is decomposed
 * independently, M_x = U_x diag(S_x) V_x, in FP64 (one-sided Jacobi, one
 * cluster of 8 CTAs per block).  U(1) and fermion-parity tensors of rank
 * >= 2 with 1 <= nrow < rank; SU(2) tensors of rank 2 (nrow = 1; the block
 * of spin x = 2j is M_x; SYM_ERR_UNSUPPORTED for higher ranks).  SU(2)
 * values and factors follow the block normalisation of the contraction
 * (1/sqrt(2j+1) per block): S holds the dense matrix's singular values
 * sigma/sqrt(2j+1) (each standing for 2j+1 of them), and U and V are
 * sqrt(2j+1) times the orthonormal block factors, so that contracting
 * U's bond with S and V rebuilds T, and U, V are isometries densely.
 *
 * sym_svd_plan: plan the decomposition of tensors with T's structure:
 *   nblocks = number of diagonal blocks (labels x with rows and columns),
 *   nsv = sum over blocks of min(m_x, n_x) (the length of S).  The plan owns
 *   a workspace of about 2.5 (max(m,n) + min(m,n)) min(m,n) doubles per
 *   block.
 * sym_svd_blocks: per block, ascending x: x, m_x, n_x (arrays of nblocks
 *   ints; any may be NULL).
 * sym_svd_execute: decompose the FP64 blocks `T` (device, T's layout).
 *   Jacobi sweeps in FP32 choose the starting point, which is made
 *   orthogonal in FP64 (Newton-Schulz); FP64 sweeps then converge to FP64
 *   accuracy, so the result is an FP64 SVD.
 *   S (device, nsv doubles, caller-owned) receives every block's singular
 *   values in descending order, blocks in ascending x; the singular vectors
 *   stay in the plan's workspace until the next execute.  Asynchronous; a
 *   block that has not converged after 64 FP64 sweeps sets the device error word
 *   (SYM_ERR_NUMERIC, see sym_device_status).
 * sym_svd_stats: per block of the last execute (ascending x; either array
 *   may be NULL): the sweeps it took and the rotations it applied, of the
 *   FP64 sweeps (fp32 = 0; the last one rotated no pair by more than 1e-8
 *   of its columns' norms, so what it left is at the FP64 rounding level)
 *   or of the FP32 sweeps (fp32 = 1; the last one rotated no pair by more
 *   than 1e-4, or it is the 40th).  Synchronizes the device.
 * sym_svd_truncation: keep[b] from a host copy of execute's S (reading of
 *   the truncation the thesis leaves open): every singular value sorted in
 *   descending order (ties: smaller x first, then the block's own order);
 *   the leading ones are kept while their dense count (SU(2): 2j+1 each,
 *   else 1) stays <= chi (chi < 0: no limit) and, if cutoff > 0, while
 *   they exceed cutoff times the largest.
 *   SYM_ERR_NUMERIC if a value is negative or not finite.  Host only.
 * sym_svd_bond: keep[b] (0 <= keep[b] <= min(m_x, n_x), blocks in ascending
 *   x, at least one > 0) singular vectors per block.  Returns the structures
 *   of U (legs: the row legs, then the bond leg, incoming; total 0) and V
 *   (legs: the bond leg, outgoing, then the column legs; T's total); the
 *   bond leg lists the labels x with keep > 0, degeneracy keep.  The caller
 *   destroys both.  Host work and one upload; later factors calls use it.
 * sym_svd_factors: write U's and V's blocks (device, FP64, the layouts of
 *   sym_svd_bond's structures) from the last execute: U's block (rows of row
 *   tuple, x) = those rows of U_x's first keep columns, V's block (x, column
 *   tuple) = those columns of V_x's first keep rows.  absorb 0: plain
 *   factors; 1: U's columns multiplied by S; 2: V's rows multiplied by S
 *   (SU(2): the orthonormal block factor times sigma).
 *   Sk (device, sum of keep doubles, may be NULL) receives the kept
 *   singular values in the bond leg's order.
 *   Where a singular value is zero, the vector obtained by dividing by it
 *   (U's column if m_x >= n_x, else V's row) is written as zeros; the
 *   product U_x diag(S_x) V_x is unchanged.  Asynchronous.                  */
typedef struct sym_svd_s* sym_svd;
int sym_svd_plan(sym_tensor T, int nrow, sym_svd* out, int* nblocks, int64_t* nsv);
int sym_svd_blocks(sym_svd plan, int* x, int* m, int* n);
int sym_svd_execute(sym_svd plan, const double* T, double* S, void* stream);
int sym_svd_stats(sym_svd plan, int fp32, int* sweeps, int64_t* rotations);
int sym_svd_truncation(sym_svd plan, const double* S, int64_t chi, double cutoff, int* keep);
int sym_svd_bond(sym_svd plan, const int* keep, sym_tensor* U, sym_tensor* V);
int sym_svd_factors(sym_svd plan, int absorb, double* U, double* V, double* Sk, void* stream);
int sym_svd_destroy(sym_svd plan);

/* --------------------------------------- blockwise eigendecomposition (FP64) ---
 * Spectral decomposition of a symmetric tensor seen as a square matrix
 * (Ch. 5, "Factorization of a matrix", Eq. spectral; the thesis obtains it,
 * like the SVD of Eq. svd0 / svd1, by factorizing every diagonal block on its
 * own).  Rows = legs 0..nrow-1, columns = legs nrow..2 nrow-1, which must be
 * the row legs reversed (same labels and degeneracies, opposite directions,
 * same order; SYM_ERR_INCOMPATIBLE_LEGS otherwise) with total label 0
 * (U(1), fermion parity), or an SU(2) tensor of rank 2 with one incoming and
 * one outgoing leg.  The block-diagonal form is the SVD's (above); every
 * block M_x is square and is taken as symmetric: the result is the
 * eigendecomposition of (M_x + M_x^T) / 2 = Q diag(lambda) Q^T.  The kernel
 * is the SVD's one-sided Jacobi applied to (M_x + M_x^T) / 2 + sigma I with
 * sigma its Frobenius norm (a positive semidefinite matrix, whose singular
 * vectors are its eigenvectors); lambda = singular value - sigma, so the
 * eigenvalues carry an absolute error of a few ulp of sigma.  SU(2): the
 * dense matrix is the direct sum of sgn_j M_x / sqrt(2j+1) (x) 1_{2j+1}, with
 * sgn_j = (-1)^{2j} if the row leg is incoming, else 1; lambda reports the
 * dense eigenvalues sgn_j lambda_x / sqrt(2j+1) (each standing for 2j+1 of
 * them) and the factors are U = sqrt(2j+1) Q, V = sgn_j sqrt(2j+1) Q^T, so
 * that U diag(lambda) V rebuilds T through the library's contraction and U
 * is an isometry densely whose columns are the dense eigenvectors.
 *
 * sym_eig_plan: as sym_svd_plan; nev = sum over blocks of m_x.  The plan is
 *   a sym_svd handle: sym_svd_blocks, sym_svd_stats, sym_svd_bond,
 *   sym_svd_factors and sym_svd_destroy apply to it unchanged (U = the
 *   eigenvectors with an incoming bond leg, V = their transposes with an
 *   outgoing bond leg; absorb 1 / 2 multiplies lambda into U / V).
 * sym_eig_execute: lambda (device, nev doubles, caller-owned) receives every
 *   block's eigenvalues ordered by |lambda| descending (ties: the larger
 *   lambda first, then the Jacobi column), blocks in ascending x.  Errors and
 *   asynchrony as sym_svd_execute.
 * sym_eig_truncation: keep[b] from a host copy of lambda: the rule of
 *   sym_svd_truncation applied to |lambda| (the singular values of a
 *   symmetric matrix), so that a truncation to chi keeps the best
 *   approximation of that rank (Eckart-Young).  Host only.               */
int sym_eig_plan(sym_tensor T, int nrow, sym_svd* out, int* nblocks, int64_t* nev);
int sym_eig_execute(sym_svd plan, const double* T, double* lambda, void* stream);
int sym_eig_truncation(sym_svd plan, const double* lambda, int64_t chi, double cutoff, int* keep);

#ifdef __cplusplus
}
#endif
#endif /* SYMTENSOR_H */
