/*
 * e2.h -- C ABI of the B300 (sm_103a) library for the Epstein-Nesbet
 * second-order energy of a multiconfigurational four-component reference.
 *
 * What it computes (Sec. 2.3, Eq. pt2; Sec. 2.4, Eq. pt2en):
 *
 *   E2_m = sum_{K in Q} |<K|H|Psi_m>|^2 / (E0_m - H_KK)
 *
 * with the Epstein-Nesbet zeroth-order Hamiltonian H0 = PHP + diag(QHQ)
 * (Eq. zeroh), Psi_m = sum_L c_{m,L} |L> over the reference space P
 * (Sec. 2.3), E0_m = <Psi_m|H|Psi_m>/<Psi_m|Psi_m>, and Q = every determinant
 * outside P that is a single or double substitution of a P determinant
 * (Sec. 2.3), restricted by frozen core / frozen virtual spinors (Sec. 2.5).
 * With b > 0 the denominator takes the imaginary level shift of Sec. 2.6 and
 * the library returns the real part: |V|^2 D^3 / (D^4 + b^2), D = E0 - H_KK.
 *
 * Hamiltonian (second quantisation over Kramers-unrestricted spinors):
 *   H = sum_pq h_pq a+_p a_q + 1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r,
 *   <pq||rs> = (pr|qs) - (ps|qr),
 *   (pq|rs)  = sum_{L in Coulomb set} B^L_pq B^L_rs
 *            + lambda * sum_{L in extra set} w_L B^L_pq B^L_rs,
 * where the extra set is the Gaunt (DCG) or Breit (DCB) factor set
 * (Sec. 2.1, Eqs. dcb, Coulomb, breit); DC has no extra set.
 *
 * Spinor order: [core | active | virtual]; frozen core spinors are always
 * occupied, frozen virtual spinors always empty.  A determinant is the
 * product of creators in ascending spinor order acting on the vacuum.
 *
 * Active space: n_das subspaces of consecutive active spinors (a CAS is one
 * subspace); P holds the active strings of n_elec electrons whose per-subspace
 * counts n_s satisfy das_min[s] <= n_s <= das_max[s] (Sec. 2.4, Eq. DASK).
 *
 * Reference coefficient order (the "address" of a P determinant): allowed
 * occupation patterns (n_1..n_k) in lexicographic order, n_1 most
 * significant, one block per pattern; inside a block
 *   sum_s rank_s * stride_s,  stride_1 = 1, stride_{s+1} = stride_s * C(size_s, n_s),
 * rank_s = colex rank of the subspace-s substring: sum_j C(t_j, j) over its
 * occupied local indices t_1 < t_2 < ... (j from 1).  For a CAS this is the
 * colex rank of the active string.
 *
 * External classes: class id = 3*h + p, h = correlated core holes (0..2),
 * p = correlated virtual particles (0..2).  Class 0 (pure active
 * rearrangement into a non-reference pattern) exists only with n_das > 1.
 *
 * Memory and ownership: every array argument is caller-owned.  Device
 * pointers must stay valid until the stream reaches the end of the call's
 * work.  The library keeps only host-side plans inside an e2_problem.  It
 * allocates no device memory: it works in the caller's workspace, of at least
 * e2_workspace_size() bytes, 256-byte aligned.
 *
 * Complex numbers are interleaved (re, im) doubles.  Arithmetic: by default
 * every step runs in IEEE FP64 (the dense contractions as complex FP64
 * products on the FP64 tensor pipe, mma.sync f64; denominators, reciprocals
 * and sums in FP64).  e2_set_contraction opts parts of the path into an
 * emulated form (bf16 slices on the tensor pipe, float-float epilogues) that
 * is faster but not FP64 arithmetic; see there.
 *
 * Errors: argument errors return immediately with a status and enqueue no
 * work.  No C++ exception crosses this interface.  Calls on one e2_problem
 * must not overlap (a problem is not thread-safe).
 */
#ifndef E2_H
#define E2_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define E2_API __attribute__((visibility("default")))
#else
#define E2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { E2_DC = 0, E2_DCG = 1, E2_DCB = 2 } e2_hamiltonian;

typedef enum {
  E2_OK = 0,
  E2_ERR_INVALID_ARG = 1,
  E2_ERR_SHAPE = 2,
  E2_ERR_UNSUPPORTED = 3,
  E2_ERR_WORKSPACE = 4,
  E2_ERR_CUDA = 5,
  E2_ERR_NONFINITE = 6,  /* device-detected: a non-finite energy (e2_query_status) */
  E2_ERR_INTRUDER = 7,   /* device-detected: |E0 - H_KK| < 1e-12 Eh with b = 0 (e2_query_status; Sec. 2.6) */
  E2_ERR_OOM = 8,        /* host memory for a plan could not be allocated */
  E2_ERR_TIMEOUT = 9     /* reserved for bounded device waits; no kernel of this version waits on another */
} e2_status;

#define E2_NCLASS 9
#define E2_MAX_DAS 8

/* Problem description (host memory; copied by e2_problem_create). */
typedef struct {
  int32_t n_core;          /* core spinors, frozen ones included (even) */
  int32_t n_active;        /* active spinors, 1..62 */
  int32_t n_virt;          /* virtual spinors, frozen ones included */
  int32_t n_elec;          /* active electrons in P */
  const uint8_t* frozen;   /* [n_core+n_active+n_virt], 1 = frozen; only core or virtual spinors may be frozen */
  int32_t n_das;           /* 1..E2_MAX_DAS active subspaces */
  const int32_t* das_size; /* [n_das], sums to n_active */
  const int32_t* das_min;  /* [n_das] minimum electrons per subspace in P */
  const int32_t* das_max;  /* [n_das] maximum electrons per subspace in P */
  int32_t ham;             /* e2_hamiltonian */
  int32_t L_coulomb;       /* Coulomb factor count (>= 1) */
  int32_t L_extra;         /* Gaunt / Breit factor count (0 for DC) */
  int32_t n_roots;         /* reference states, 1..16 */
  double level_shift_b;    /* b >= 0 of the imaginary level shift; 0 = plain Eq. pt2 */
  uint32_t class_mask;     /* bit c: evaluate class c (3h+p); 0x1FF = all */
} e2_desc;

/* Device inputs of one evaluation.  All device pointers, complex interleaved:
 *   h   [n][n]           Hermitian one-electron matrix
 *   B_c [L_coulomb][n][n] Hermitian Coulomb factors
 *   B_x [L_extra][n][n]   Hermitian Gaunt/Breit factors (NULL if L_extra == 0)
 *   w_x [L_extra]         real weights of the extra factors (NULL if L_extra == 0)
 *   c   [n_roots][N_P]    reference coefficients in address order (need not be normalised)
 */
typedef struct {
  const double* h;
  const double* B_c;
  const double* B_x;
  const double* w_x;
  double lambda;           /* multiplier of the extra set (1 = full Gaunt/Breit) */
  const double* c;
} e2_inputs;

typedef struct e2_problem e2_problem;

/* Validates the description and builds the host plan (occupation patterns,
 * string-list sizes, workspace layout).  No device work.  *out is NULL on error. */
E2_API e2_status e2_problem_create(const e2_desc* desc, e2_problem** out);
E2_API e2_status e2_problem_destroy(e2_problem* prob);

/* N_P, and the number of external determinants per class (|Q| split by
 * class id, per root), both as computed by the plan. */
E2_API e2_status e2_problem_info(const e2_problem* prob, int64_t* n_p, double* q_per_class /* [E2_NCLASS] or NULL */);

/* Device workspace needed by e2_forward. */
E2_API e2_status e2_workspace_size(const e2_problem* prob, size_t* bytes);

/* E2 for every root.  Enqueues kernels on `stream` (a cudaStream_t; NULL = the
 * legacy default stream) and returns without synchronising.
 *   E2       device [n_roots]            total second-order energy per root
 *   E2_class device [n_roots][E2_NCLASS]  per-class contributions, or NULL
 *   E0       device [n_roots]            reference energies, or NULL
 * The summation order is fixed, so repeated calls give bitwise equal results. */
E2_API e2_status e2_forward(e2_problem* prob, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                     void* stream, double* E2, double* E2_class, double* E0);

/* Coupling tensors of one reference state (step a4: the <K|E_pq|L> C_L
 * factors of Sec. 2.4, Eq. sumsigma, restricted to the active space), for
 * inspection.  Builds the string lists and root `root`'s tables in
 * `workspace` as e2_forward does, then copies one family:
 *   family 0  D^t_A     = <A|a_t|Psi>,             rows t (n_act);          strings of N-1 electrons (class (1,2))
 *          1  D^{t+}_A  = <A|a+_t|Psi>,            rows t;                  N+1 (class (2,1))
 *          2  D^{tu}_A  = <A|a_u a_t|Psi>, t < u,  row u(u-1)/2 + t;        N-2 (class (0,2))
 *          3  D^{t+u+}_A = <A|a+_t a+_u|Psi>, t < u, same rows;            N+2 (class (2,0))
 *          4  row 0: c_A; row 1 + t n_act + u: <A|a+_t a_u|Psi>;            N   (class (1,1))
 *   table   device [rows][n_A] complex, or NULL
 *   strings device [n_A] active-local bitsets (bit t = active spinor t) of
 *           the class's string list in address order, or NULL
 *   rows, n_A host, or NULL: the table's shape (both outputs NULL: sizes
 *           only, no device work)
 * Every entry is exactly +-c_L of one P determinant L or 0.  Enqueues on
 * `stream`; inputs and workspace as for e2_forward.  E2_ERR_INVALID_ARG for
 * a family or root out of range. */
E2_API e2_status e2_coupling_tables(e2_problem* prob, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                                   void* stream, int root, int family, double* table, uint64_t* strings,
                                   int64_t* rows, int64_t* n_A);

/* Per-coupling probe (no counterpart in the paper; it lets a caller check
 * single couplings V_K = <K|H|Psi> and D_K = E0 - H_KK of a full-size run
 * against an independent evaluation).  Sets up root `root` as e2_forward
 * does, then runs the FP64 class kernel of class cls (the same device code as
 * the forward's, whatever arithmetic the class is set to) with its probe
 * outputs on:
 *   dense classes (0,2) (1,2) (1,1) (2,0) (2,1): the 64 x 64 tile (tile_m,
 *     tile_n) as e2_partials numbers tiles; V device [64][64] complex, D
 *     device [64][64]; entry [i][j]: external row 64 tile_m + i (the row
 *     order of e2_partials), string = column j of the tile (plain columns:
 *     list index 64 tile_n + j; column tiles: perm[64 tile_n + j] of
 *     e2_class_tiles_copy); entries outside the class are 0;
 *   gather classes (0,1) (1,0) (0,0): the whole class; tile_m, tile_n
 *     ignored; V device [rows][n_A] complex, D device [rows][n_A], rows = the
 *     correlated virtuals (0,1), the correlated core spinors (1,0) or one row
 *     (0,0), strings in the class list's address order.
 *   shape host [2] or NULL: the shape of V and D; with V and D both NULL
 *     only the shape is returned (no device work).
 * V is formed from the unnormalised c (as the partials are).  Class (2,2)
 * (elementwise, V = <ab||ij> c_A up to sign, never formed) returns
 * E2_ERR_UNSUPPORTED, as does a class without couplings.  Enqueues on
 * `stream`; inputs and workspace as for e2_forward (the probe writes the
 * tile's partial slot too). */
E2_API e2_status e2_probe_couplings(e2_problem* prob, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                                   void* stream, int root, int cls, int64_t tile_m, int64_t tile_n, double* V,
                                   double* D, int64_t* shape);

/* Intruder diagnostics (Sec. 2.6): how close the denominators D = E0 - H_KK
 * of root `root` come to zero, per class, as a histogram by decades:
 *   hist device [E2_NCLASS][E2_DHIST] uint64 (overwritten): bin 0 counts
 *     |D| < 1e-12 Eh (intruder states when b = 0), bin k = 1..16 counts
 *     10^(k-13) <= |D| < 10^(k-12) Eh, bin 17 the rest (|D| >= 1e4 Eh or NaN).
 * Every external determinant of every evaluated class counts once (class
 * (2,2) also where <ab||ij> vanishes), so row c sums to the class's size.
 * A diagnostic pass: it sets up root `root` as e2_forward does and evaluates
 * every denominator (no V).  Enqueues on `stream`; inputs and workspace as
 * for e2_forward. */
#define E2_DHIST 18
E2_API e2_status e2_denominator_histogram(e2_problem* prob, const e2_inputs* in, void* workspace,
                                          size_t workspace_bytes, void* stream, int root, unsigned long long* hist);

/* Integral formation alone (step a5; the paper's AO -> MO transformation,
 * T_int of Sec. 3.1 Table 1, here from the factors B^L): everything of
 * e2_forward that depends only on the Hamiltonian and the partition -- the
 * compact factor block, G, eps^, f^(O), the string lists with e_A and U, and
 * every integral block the classes contract: <ab||tu>, <ab||it>, <at||ij>,
 * <at||iu> with f^(O)_ai, <tu||ij>, |<ab||ij>|^2, <au||vw>, <tu||iv>,
 * <tu||vw> -- into `workspace`, then stops.  c is not read (may be NULL).
 * Enqueues on `stream`; workspace as for e2_forward. */
E2_API e2_status e2_form_integrals(e2_problem* prob, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                                   void* stream);

/* Sharding of the external space over ranks (no counterpart in the paper's
 * method; its sigma-build is distributed over CPU nodes, Sec. 2.4 / 3.1, which
 * is prior art here).  Every class's work is cut into units -- row tiles of a
 * dense class, (core pair, 8-wide virtual block pair) units of (2,2), rows
 * (virtual a / core i) of (0,1) / (1,0), 256-string blocks of (0,0) -- and
 * rank r of n takes the contiguous units [u r / n, u (r+1) / n) of each class.
 * Everything else (integrals, string lists, coupling tables, E0) is
 * replicated.  A sharded e2_forward writes only its own partial slots and
 * zeroes the others, so the element-wise sum of all ranks' partials is
 * bit for bit the unsharded set:
 *   e2_set_shard(prob, rank, n);  e2_forward(...);
 *   (caller) sum the partials over ranks (e2_shard_buffers gives the device
 *            array; e.g. an all-reduce SUM) and take the minimum of the |D|
 *            keys (int64, same call; all-reduce MIN);
 *   e2_reduce(prob, workspace, ...)  -> E2, E2_class, E0 of the whole space,
 *            bitwise equal to an unsharded e2_forward for any n.
 * The E2 output of a sharded e2_forward is this rank's share alone.
 * e2_backward and e2_batch_forward return E2_ERR_UNSUPPORTED on a sharded
 * problem; e2_set_shard(prob, 0, 1) undoes the split.
 *   e2_shard_units   units of class cls and this rank's [first, end)
 *   e2_shard_buffers device pointers into `workspace`: the partials
 *                    (n_partials doubles, all roots and classes) and the
 *                    smallest-|D| keys (n_keys int64, ordered like |D|) */
E2_API e2_status e2_set_shard(e2_problem* prob, int rank, int n_ranks);
E2_API e2_status e2_shard_units(const e2_problem* prob, int cls, int64_t* units, int64_t* first, int64_t* end);
E2_API e2_status e2_shard_buffers(const e2_problem* prob, void* workspace, double** partials, int64_t* n_partials,
                                  int64_t** min_keys, int64_t* n_keys);
E2_API e2_status e2_reduce(e2_problem* prob, void* workspace, size_t workspace_bytes, void* stream, double* E2,
                           double* E2_class, double* E0);
/* What e2_reduce reads besides the partials -- every root's E0 and <c|c> --
 * set up in `workspace` without any class work (setup and the coupling
 * tensors of each root in turn).  With it, partial sets saved piece by piece
 * (each piece a shard's e2_forward, its partials written to a file) can be
 * summed back into the workspace by a later process and reduced: a long run
 * resumes where it stopped, with the result bitwise equal to the unsharded
 * forward (checkpoint / resume). */
E2_API e2_status e2_prepare_roots(e2_problem* prob, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                                  void* stream);

/* Device status word (the conditions of Sec. 2.6 that only the device sees).
 * Every e2_forward (also e2_forward_noalloc, each job of e2_batch_forward and
 * e2_backward with an E2 output) clears it at its start and writes it in its
 * workspace; e2_query_status reads it back after that work:
 *   flags     bit E2_STATUS_NONFINITE: some class energy or E2 is NaN or
 *             infinite (a non-finite input propagates into it; on the sliced
 *             path the slicers turn a non-finite operand into a NaN scale);
 *             bit E2_STATUS_INTRUDER: with b = 0, some external determinant
 *             of an evaluated class has |E0 - H_KK| below 1e-12 Eh (an
 *             intruder state; the imaginary level shift b > 0 of Sec. 2.6 is
 *             the remedy).  May be NULL.
 *   min_abs_D host [n_roots][E2_NCLASS] or NULL: the smallest |E0 - H_KK| over
 *             the couplings of each class (+inf for a class without couplings;
 *             class (2,2): over its couplings with non-zero <ab||ij>).
 * Returns E2_ERR_NONFINITE if that flag is set, else E2_ERR_INTRUDER if that
 * one is, else E2_OK; E2_ERR_CUDA if the read fails.  Synchronises `stream`
 * (the copy is enqueued on it); `workspace` is the one the work used (for
 * e2_forward_noalloc pass NULL: the library's own scratch). */
#define E2_STATUS_NONFINITE 1u
#define E2_STATUS_INTRUDER 2u
E2_API e2_status e2_query_status(const e2_problem* prob, const void* workspace, void* stream, uint32_t* flags,
                                 double* min_abs_D);

/* Batches (no counterpart in the paper: a throughput device).  Several
 * planned problems -- different Hamiltonians, root counts, frozen cutoffs,
 * CAS or DAS references -- evaluated together: every class of every job and
 * root (the dense-class tiles, the (2,2) blocks and the gather-class blocks)
 * runs in ONE persistent launch, one CTA per SM, that takes work items from
 * an integer counter, longest item first; only the per-job set-up before it
 * and the reductions after it are separate launches (and the classes a job
 * opted into the emulated arithmetic, which keep their own kernels).  Results
 * equal those of e2_forward job by job (same partial slots, same fixed
 * reduction order).  Every root of every job keeps its coupling tables until
 * the one launch, so the workspace grows with the roots (e2_batch_workspace_size).
 *   e2_batch_create   host only; the problems must outlive the batch.
 *   e2_batch_prepare  uploads plan tables and the work list into `workspace`
 *                     and synchronises `stream`; call it once per workspace,
 *                     outside stream capture.
 *   e2_batch_forward  kernels, memsets and device-to-device copies only (no
 *                     host synchronisation, no host-to-device copies): it can
 *                     be captured in a CUDA graph and replayed.  `workspace`
 *                     must be the prepared one.
 *                     inputs [n_jobs]; E2 [n_jobs] device pointers ([n_roots_j]
 *                     each); E2_class [n_jobs] or NULL. */
typedef struct e2_batch e2_batch;
E2_API e2_status e2_batch_create(e2_problem* const* jobs, int n_jobs, e2_batch** out);
E2_API e2_status e2_batch_destroy(e2_batch* batch);
E2_API e2_status e2_batch_workspace_size(const e2_batch* batch, size_t* bytes);
E2_API e2_status e2_batch_prepare(e2_batch* batch, void* workspace, size_t workspace_bytes, void* stream);
E2_API e2_status e2_batch_forward(e2_batch* batch, const e2_inputs* inputs, void* workspace, size_t workspace_bytes,
                                  void* stream, double* const* E2, double* const* E2_class);
E2_API e2_status e2_batch_launch_count(const e2_batch* batch, int64_t* n);
/* Root groups: with k > 0, the batch runs its roots in groups -- roots
 * 0..k-1 of every job in the first persistent launch, k..2k-1 in the next --
 * and keeps only k coupling-table slots per job (root r in slot r mod k),
 * rebuilt before each launch; k = 0 (the default) runs every root in one
 * launch.  This bounds the workspace when the tables of all job-roots do not
 * fit the device together (at a CAS(8e,24) active space one root's tables
 * take about 17 GB).  Results are unchanged (bitwise).  Host only; call it
 * before e2_batch_workspace_size and e2_batch_prepare (it re-lays the
 * workspace). */
E2_API e2_status e2_batch_set_roots_per_launch(e2_batch* batch, int k);
/* Adjoint of a batch: each job's e2_backward in turn, in one workspace of
 * e2_batch_backward_workspace_size() bytes (the largest job's backward
 * layout; the forward batch's prepared workspace is not needed).  Per job j:
 * seeds[j] host [n_roots_j]; g_h, g_c, g_Bc, g_Bx, dE2_dlambda, E2: arrays of
 * n_jobs device pointers as e2_backward takes them (an array, or an entry,
 * may be NULL to skip that output).  The energies are bitwise equal to
 * e2_forward's and e2_batch_forward's of the same job.  The passes are
 * enqueued one after another on `stream` (not merged into one launch). */
E2_API e2_status e2_batch_backward_workspace_size(const e2_batch* batch, size_t* bytes);
E2_API e2_status e2_batch_backward(e2_batch* batch, const e2_inputs* inputs, const double* const* seeds,
                                  void* workspace, size_t workspace_bytes, void* stream, double* const* g_h,
                                  double* const* g_c, double* const* g_Bc, double* const* g_Bx,
                                  double* const* dE2_dlambda, double* const* E2);

/* Adjoint of e2_forward (gradients are not in the paper; they follow from
 * differentiating Eq. pt2 with E0 = <Psi|H|Psi>/<Psi|Psi>).  For
 * F = sum_m seed[m] E2_m it returns, for complex inputs z, dF/dRe z + i dF/dIm z:
 *   g_h  device [n][n]          projected on Hermitian matrices (the unrelaxed
 *                               response one-particle density), or NULL
 *   g_c  device [n_roots][N_P]  gradient for each root's coefficients, or NULL
 *                               (orthogonal to c: E2 does not depend on |c|)
 *   g_Bc device [L_coulomb][n][n], g_Bx device [L_extra][n][n]
 *                               factor gradients, Hermitian-projected, or NULL
 *   dE2_dlambda device [1]      dF/dlambda: the Gaunt / Breit share of the
 *                               correlation energy to first order, or NULL
 *   seed host [n_roots]
 *   E2   device [n_roots], or NULL: the energies themselves, bitwise equal to
 *        e2_forward's (the pass forms every V anyway), so that one call gives
 *        the value and its gradient
 * V is recomputed (never stored whole): the dense classes run in row chunks
 * whose weighted amplitudes fit 4 GiB (and whose compacted Gamma_W, for a
 * column-tiled class, fits 8 GiB); class (2,2) runs in chunks of core pairs
 * whose partial sums fit 2 GiB.  Enqueues on `stream`; workspace of at least
 * e2_backward_workspace_size() bytes (it contains the e2_forward and
 * reference-solver layouts). */
E2_API e2_status e2_backward_workspace_size(const e2_problem* prob, size_t* bytes);
E2_API e2_status e2_backward(e2_problem* prob, const e2_inputs* in, const double* seed, void* workspace,
                             size_t workspace_bytes, void* stream, double* g_h, double* g_c, double* g_Bc,
                             double* g_Bx, double* dE2_dlambda, double* E2);
/* Smaller adjoint chunks than the plan's (the workspace layout is unchanged):
 * rows per dense-class chunk (rounded down to a multiple of 64, at least 64)
 * and core pairs per class-(2,2) chunk, each capped at the plan's value; 0
 * (or less) restores the plan's value.  The results change only by the order
 * of the sums across chunks.  E2_ERR_INVALID_ARG for a NULL problem. */
E2_API e2_status e2_set_adjoint_chunks(e2_problem* prob, int64_t rows, int core_pairs);

/* Reference states: the n_roots lowest eigenvectors of P H P (the CASCI /
 * DAS-CI reference of Sec. 2.2-2.3, Eq. zeroh first term), by block Davidson
 * iteration on the device (sigma = P H c built from the same coupling
 * tensors as the (0,0) class; preconditioner diag(H_PP)).  Convergence: every
 * residual norm ||H x - theta x|| < tol for unit-norm x.
 *   in->c     device [n_roots][N_P] start vectors (any full-rank block)
 *   c_out     device [n_roots][N_P] unit-norm eigenvectors (may alias in->c)
 *   E0_out    host   [n_roots] eigenvalues, ascending
 *   iters_out host, iterations used (may be NULL)
 * Synchronises `stream` (small projected problems are solved on the host).
 * Returns E2_ERR_SHAPE if the start block is rank deficient.  The workspace
 * must be at least e2_reference_workspace_size() bytes (it contains the
 * e2_forward layout). */
E2_API e2_status e2_reference_workspace_size(const e2_problem* prob, size_t* bytes);
E2_API e2_status e2_reference_solve(e2_problem* prob, const e2_inputs* in, double tol, int max_iter, void* workspace,
                                    size_t workspace_bytes, void* stream, double* c_out, double* E0_out, int* iters_out);

/* Measurement hooks (no counterpart in the paper; used for the roofline).
 * e2_profile_events: `events` is NULL (off) or 2*E2_NCLASS cudaEvent_t
 * handles owned by the caller; e2_forward then records events[2c] before and
 * events[2c+1] after the class-c kernel of root 0 on its stream.
 * e2_fp64_peak: times FP64 tensor-pipe (mma.sync m16n8k8 f64) and FP64 FMA
 * throughput on the current device in TFLOP/s.  Needs a device scratch of
 * 8 * 256 * 8 * (SM count) bytes; synchronises `stream`. */
E2_API e2_status e2_profile_events(e2_problem* prob, void* const* events);
/* Number of kernels the last e2_forward on this problem enqueued. */
E2_API e2_status e2_launch_count(const e2_problem* prob, int64_t* n);
E2_API e2_status e2_fp64_peak(void* workspace, size_t workspace_bytes, void* stream, double* dmma_tflops,
                              double* dfma_tflops);

/* Per-CTA partial sums of the last e2_forward (or e2_backward with E2) that
 * used `workspace` (no counterpart in the paper; it lets a caller check any
 * block of couplings of a full-size run against an independent evaluation).
 * Sets *partials to a device pointer into the workspace (valid until the
 * workspace is reused) and *count to the number of partials of (root, cls),
 * cls = 3 h + p.  Each partial is sum |V_K|^2 g(D_K) over its couplings, with
 * V from the unnormalised c (E2 divides the total by <c|c>), g = 1/D or the
 * level-shifted weight.  Layout:
 *   dense classes (0,2) (1,2) (1,1) (2,0) (2,1): 64 x 64 tiles of (external
 *     row, class string), partial[tile_n * row_tiles + tile_m]; rows in the
 *     class's row order (pairs a<b of correlated virtuals have index
 *     b(b-1)/2 + a; (i, a<b) is i * npair_v + pair(a,b); (i<j, a) is
 *     pair(i,j) * n_vc + a; (i, a) is i * n_vc + a; (i<j) is pair(i,j)),
 *     strings of the class's list in address order (the convention at the
 *     top of this file, over the occupation patterns the class reaches);
 *   gather classes (0,1) (1,0) (0,0): per row (virtual a, core i, or the
 *     single row) blocks of 256 strings, partial[row * ceil(n_A/256) + block];
 *   class (2,2): kernel order; *row_tiles = 0 for every non-dense class.
 * columns: see the column tiles below (NULL output allowed).
 * Errors: E2_ERR_INVALID_ARG for a NULL argument or root / cls out of range. */
E2_API e2_status e2_partials(const e2_problem* prob, const void* workspace, int root, int cls,
                             const double** partials, int64_t* count, int64_t* row_tiles,
                             const int32_t** columns);

/* Column tiles of the dense classes (no counterpart in the paper; a layout
 * choice).  The coupling tables D^{tu} (class (0,2)), D^{t+u+} (class (2,0))
 * and D^{t+u} (class (1,1)) are mostly structural zeros: D^{tu}_A = 0
 * whenever t or u is occupied in A.  The plan groups the class's strings
 * into 64-column tiles whose strings share three occupied (or empty)
 * spinors, and each tile contracts only over the table rows that are
 * non-zero for one of its strings.  The result is the same sum in a
 * different order.
 *   e2_class_tiles     tiles, compacted rows (sum over tiles of the padded
 *                      contraction length) and whether class cls uses them; 0
 *                      tiles when the class has no such plan.
 *   e2_set_class_tiles switch a class to compacted (on = 1) or plain
 *                      columns; E2_ERR_UNSUPPORTED when it has no plan.  The
 *                      plan's default: on when the compacted work is below
 *                      85% of the plain work.
 *   e2_autotune        times the class kernel of root 0 both ways for every
 *                      class that has a plan and keeps the faster.  ms_out
 *                      [2 * E2_NCLASS] (host, or NULL) receives the plain and
 *                      compacted times.  It synchronises `stream`; workspace
 *                      as for e2_forward, inputs as for e2_forward.
 * When a class uses column tiles, e2_partials' tile_n indexes the column
 * tiles and *columns (device, [tiles * 64]) gives each tile column's string
 * (list index, -1 for padding); otherwise *columns is NULL. */
E2_API e2_status e2_class_tiles(const e2_problem* prob, int cls, int64_t* tiles, int64_t* krows, int* in_use);
/* The plan's column tiles of class cls as host copies, for inspection: perm
 * [tiles * 64] (list index per tile column, -1 padding), tdesc [tiles * 4]
 * ({koff, klen, ktrue, 0} per tile) and klist [krows] (table row of each
 * compacted row); sizes from e2_class_tiles.  E2_ERR_UNSUPPORTED when the
 * class has no plan. */
E2_API e2_status e2_class_tiles_copy(const e2_problem* prob, int cls, int32_t* perm, int32_t* tdesc, int32_t* klist);
E2_API e2_status e2_set_class_tiles(e2_problem* prob, int cls, int on);
/* Tuning cache for e2_autotune's choices (no counterpart in the paper): a text
 * file of lines "<key> | <column-tile choice of the nine classes>", the key
 * made of every plan input that shapes the classes (spinor counts, DAS
 * partition, frozen spinors, factor counts, roots, class mask).
 *   e2_tuning_save appends this problem's current choices (E2_ERR_INVALID_ARG
 *                  when the file cannot be written);
 *   e2_tuning_load applies the last line whose key matches; E2_ERR_UNSUPPORTED
 *                  when the file is missing or holds none (the plan's
 *                  defaults then stay). */
E2_API e2_status e2_tuning_save(const e2_problem* prob, const char* path);
E2_API e2_status e2_tuning_load(e2_problem* prob, const char* path);

/* Arithmetic of the dense-class contraction (step a7; no counterpart in the
 * paper, which computes in FP64).  The default everywhere is FP64.
 *   E2_CONTRACT_FP64   complex FP64 products on the FP64 tensor pipe
 *                      (mma.sync f64), plain or column-tiled, FP64 epilogue.
 *                      The default for every class and product.
 *   E2_CONTRACT_SLICED opt-in emulation, NOT FP64 arithmetic: the slicing of
 *                      Ozaki et al.: five 8-bit slices of each operand on the
 *                      bf16 tensor pipe with exact FP32 accumulation of the
 *                      leading levels, and the Epstein-Nesbet epilogue in
 *                      float-float arithmetic (each V to about 2^-40 of its
 *                      row and string scale; about 48 significant bits in the
 *                      epilogue; class energies within about 1e-11 relative of
 *                      the FP64 ones on the tested shapes).  Available for
 *                      (0,2), (1,2), (2,1), (2,0) when the real contraction
 *                      length 2 K is at most 256 and the slices fit 16 GiB.
 * For class (2,2) (cls 8, elementwise, no contraction) E2_CONTRACT_SLICED
 * selects the float-float kernel for its denominators and sums (available
 * when the float-float string tables fit the same 16 GiB).
 * cls = E2_CONTRACT_SETUP selects the same choice for the products over the
 * factor index that form the integral blocks (step a5: (ai|bt), (at|bu),
 * (av|uw)); there the slices are exact per 256 real terms and the sums over
 * the factor index accumulate in float-float.
 * cls = E2_CONTRACT_ADJOINT selects it for the products of e2_backward
 * (Gamma_D = W^T conj(T), Gamma_W = conj(T) D^T per row chunk, and
 * Cs = B Gamma^ when its slices fit 4 GiB; four slices, 2^-33 of the
 * scales).  A non-finite operand of a sliced product makes the energies NaN
 * (the slicers flag it) and sets E2_ERR_NONFINITE in the status word.
 * e2_set_contraction returns E2_ERR_UNSUPPORTED for a class without the
 * sliced plan; e2_contraction reports the mode in use and whether the sliced
 * plan exists (either output may be NULL).  The backward pass forms its
 * amplitudes in FP64 either way; its E2 output comes from the forward's
 * kernel, so it stays bitwise equal to e2_forward's. */
#define E2_CONTRACT_FP64 0
#define E2_CONTRACT_SLICED 1
#define E2_CONTRACT_SETUP (-1)
#define E2_CONTRACT_ADJOINT (-2)
E2_API e2_status e2_set_contraction(e2_problem* prob, int cls, int mode);

/* DAS subspaces in the core and virtual spaces (Sec. 2.4, Fig. 1: the core
 * and external virtual spaces partitioned into further DAS subspaces, each
 * category characterised by its occupation pattern over them) with per-
 * subspace limits on the external excitations: at most core_max_holes[s]
 * holes in core subspace s and virt_max_particles[s] particles in virtual
 * subspace s, on top of the global two holes / two particles.  Subspaces are
 * consecutive blocks of the core (sizes summing to n_core) and of the
 * virtual spinors (summing to n_virt) in global order.  A limit of 2 (or
 * more) leaves the subspace unrestricted; a limit of 0 is a frozen block and
 * is given with the frozen mask instead (E2_ERR_INVALID_ARG here).  The
 * determinants the limits exclude leave Q: they contribute nothing to E2,
 * the gradients, the status word or the histogram, and the class sizes of
 * e2_problem_info drop accordingly.  n_cdas = n_vdas = 0 removes all limits.
 * Host only; takes effect from the next call that uploads the plan. */
E2_API e2_status e2_set_external_das(e2_problem* prob, int n_cdas, const int32_t* core_size,
                                     const int32_t* core_max_holes, int n_vdas, const int32_t* virt_size,
                                     const int32_t* virt_max_particles);
E2_API e2_status e2_contraction(const e2_problem* prob, int cls, int* mode, int* sliced_available);
E2_API e2_status e2_autotune(e2_problem* prob, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                             void* stream, float* ms_out);

/* Allocation-free variant of e2_forward (no counterpart in the paper).
 * Some callers cannot call cudaMalloc: plugins living inside a host program
 * that owns the device allocator, and embedded runtimes that forbid device
 * allocation after start-up.  This entry point runs exactly the computation
 * of e2_forward, but in a scratch array compiled into the library,
 * E2_STATIC_SCRATCH_BYTES per device, which every device that loads the
 * library holds until the process exits.  It allocates nothing and takes no
 * workspace argument; inputs and outputs are the caller's, as for e2_forward.
 *   - A problem whose e2_workspace_size() exceeds E2_STATIC_SCRATCH_BYTES is
 *     rejected with E2_ERR_WORKSPACE before any GPU work.
 *   - Each call looks up the array's device address on the current device
 *     (a host-side query), so it runs on whichever device is current.
 *   - All calls, on every problem, share the one array and leave the last
 *     call's contents in it: calls whose GPU work can overlap (other streams,
 *     other host threads) overwrite each other's scratch and give wrong
 *     results; serialise them on one stream.
 *   - Like e2_forward it uploads the plan tables from host memory on every
 *     call.  Its status word lives in the same array (e2_query_status with a
 *     NULL workspace). */
#define E2_STATIC_SCRATCH_BYTES (32u << 20)
E2_API e2_status e2_forward_noalloc(e2_problem* prob, const e2_inputs* in, void* stream, double* E2,
                                    double* E2_class, double* E0);

E2_API const char* e2_status_string(e2_status s);

#ifdef __cplusplus
}
#endif

#endif /* E2_H */
