/*
 * lrugb.h -- C ABI of the GB300 library for batched low-rank updates (LRU) of
 * determinant and Pfaffian ratios and of the inverse matrix, across many
 * Monte Carlo walkers, in plain and delayed form.
 *
 * Method: arXiv 2602.05255 ("lrux"), Sec. 2 (determinants), Sec. 3
 * (Pfaffians), App. A (Pfaffian definition, identities, gradient).
 *
 * Notation used by every call (the paper writes the determinant update as
 * A_t = A_{t-1} + v u^T and the Pfaffian update as A_t = A_{t-1} - u J u^T):
 *   determinant : A' = A + U V,        U is n x k, V is k x n
 *                 R  = I_k + V A^{-1} U,          ratio = det R
 *                 A'^{-1} = A^{-1} - (A^{-1}U) R^{-1} (V A^{-1})
 *                 (Sec. 2.1, Eqs. det_R, det_ratio, det_inv)
 *   Pfaffian    : A' = A + B C B^T,    B is n x 2k, C is 2k x 2k skew
 *                 M  = C^{-1} + B^T A^{-1} B,      ratio = pf M / pf C^{-1}
 *                 (App. A.2, Eq. pf_low_rank; with C = -J this is Sec. 3.1,
 *                 Eqs. pf_ratio, pf_R)
 * All transposes are plain transposes, also for complex scalars.
 *
 * Conventions
 *   - Every data pointer is a DEVICE pointer owned by the caller unless the
 *     comment says "host".  The library owns only the per-walker state it
 *     allocates in lru_create (and frees in lru_destroy).
 *   - Calls enqueue work on the handle's stream and return after host-side
 *     validation; results are ready after the stream is synchronised.
 *   - Scalars have the handle's dtype: double, {double re, im}, float or
 *     {float re, im}.  log|value| is always double.
 *   - Matrices passed in (A) are row-major, walker after walker; with ragged
 *     sizes walker w starts at element sum_{v<w} n_v^2.
 *   - Length-n vectors (operands, one per update column) are stored walker
 *     after walker with kmax slots per walker: vector a of walker w starts at
 *     element (voff_w * kmax) + a * n_w where voff_w = sum_{v<w} n_v
 *     (uniform n: (w*kmax + a)*n).  For the Pfaffian kmax counts the 2k
 *     columns of B.
 *   - Return value: LRU_OK, or the first host-side error.  Per-walker results
 *     (singular core, non-finite ratio) go to the per-walker status array.
 *     Device-side faults of the library's own checks (bounded waits that ran
 *     out, index out of range) set a sticky handle error that
 *     lru_check_device_error reports.
 */
#ifndef LRUGB_H
#define LRUGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LRU_OK = 0,
    LRU_ERR_ARG = 1,          /* invalid argument (NULL, size, kind, dtype) */
    LRU_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    LRU_ERR_NOMEM = 3,        /* device allocation failed */
    LRU_ERR_STATE = 4,        /* call out of order (e.g. accept without propose) */
    LRU_ERR_SINGULAR = 5,     /* a matrix that must be invertible is singular */
    LRU_ERR_NOT_SKEW = 6,     /* a Pfaffian input is not skew-symmetric */
    LRU_ERR_TIMEOUT = 7,      /* a bounded device wait gave up (sticky) */
    LRU_ERR_UNSUPPORTED = 8   /* combination not built (reported, never faked) */
} lru_status;

/* per-walker status codes (int32 array written by propose / refresh) */
#define LRU_WALKER_OK 0
#define LRU_WALKER_SINGULAR 1      /* core R (or M) singular: ratio 0 is a node; accept skipped */
#define LRU_WALKER_NONFINITE 2     /* ratio or core not finite: accept skipped */
#define LRU_WALKER_BAD_INDEX 3     /* one-hot index outside [0, n) */

typedef enum { LRU_F64 = 0, LRU_C128 = 1, LRU_F32 = 2, LRU_C64 = 3 } lru_dtype;
typedef enum { LRU_DET = 0, LRU_PF = 1 } lru_kind;

/* Precision of the delayed flush A0^{-1} -/+= P Q^T (Sec. 2.3 Eq. delayed_Ainv,
 * Sec. 3.3 Eq. pf_delayed_Ainv).  Everything else stays in the handle dtype. */
typedef enum {
    LRU_FLUSH_NATIVE = 0,   /* dtype arithmetic on the CUDA cores (FP64 for F64/C128) */
    LRU_FLUSH_TF32X3 = 1,   /* tcgen05 TF32 tensor cores, 3-term split (about FP32 accuracy) */
    LRU_FLUSH_TF32 = 2,     /* tcgen05 TF32, one term */
    LRU_FLUSH_BF16 = 3,     /* tcgen05 BF16, one term */
    LRU_FLUSH_BF16X3 = 4,   /* tcgen05 BF16, 3-term split */
    LRU_FLUSH_DF = 5,       /* F64 only: double-float products on the FP32 pipe (about 1e-14 relative) */
    LRU_FLUSH_SPLIT = 6     /* F64, uniform n % 128 == 0 (n <= 2048), K*k <= 64 (Pfaffian: K*2k): exact
                               BF16 split products on the tensor cores with FP64 recombination (the
                               rounding of an FP64 update); for the Pfaffian the upper triangle of the
                               result is kept and the lower one written as its exact negative */
} lru_flush;

/* Arithmetic of the streaming passes over A^{-1} for F64 handles. */
typedef enum {
    LRU_ARITH_NATIVE = 0,   /* FP64 FMAs */
    LRU_ARITH_DF = 1        /* double-float (pairs of FP32) from integer-split FP64 data, about 2^7 x
                               FP64's rounding: the delayed GEMV of rank-1 determinant updates
                               (HBM-bound instead of FP64-bound) and the Pfaffian propose's pass.
                               For uniform-n Pfaffian handles that pass reads the inverse as exactly
                               skew ((A^-1)_jl = -(A^-1)_lj, rows streamed contiguously), which the
                               init, refresh, lru_accept and every flush keep bit for bit; after
                               lru_step_persistent's plain Pfaffian accept (a generic Woodbury
                               update, not exactly skew) refresh before such a propose */
} lru_arith;

/* How init and refresh compute the FP64 inverse (F64 determinant handles):
 * the update of each 64-column Gauss-Jordan panel on the other columns is an
 * n x n x 64 product; LRU_REFRESH_TENSOR runs it on the BF16 tensor cores as
 * an exact split product (7 slices of 8 bits per operand, FP64 recombination:
 * the accuracy of an FP64 update), the panels themselves in FP64.  It applies
 * to uniform n with n % 128 == 0, 128 <= n <= 2048 and W <= 65535; other
 * handles use LRU_REFRESH_FP64.  A refresh that asks for the drift allocates,
 * on first use, a second W x n x n workspace for the fresh inverses. */
typedef enum {
    LRU_REFRESH_AUTO = 0,     /* the tensor-core form where it applies */
    LRU_REFRESH_FP64 = 1,     /* blocked Gauss-Jordan entirely on the FP64 pipe */
    LRU_REFRESH_TENSOR = 2    /* as AUTO; lru_create fails with LRU_ERR_UNSUPPORTED where it cannot apply */
} lru_refresh;

typedef struct {
    int32_t kind;                 /* lru_kind */
    int32_t dtype;                /* lru_dtype */
    int64_t walkers;              /* W >= 1 */
    int32_t n;                    /* uniform matrix size, or 0 when n_per_walker is given */
    const int32_t* n_per_walker;  /* host, W entries, or NULL */
    int32_t k;                    /* update rank: det U has k columns; pf B has 2k columns (uniform) */
    const int32_t* k_per_walker;  /* host, W entries (each <= k), or NULL */
    int32_t delay;                /* K of the delayed form (Sec. 2.3 / 3.3); 0 or 1 = plain updates */
    int32_t flush;                /* lru_flush */
    int32_t device;               /* CUDA device ordinal */
    int32_t arith;                /* lru_arith (F64 handles; ignored otherwise) */
    int32_t tile_chunks;          /* columns of A^{-1} per CTA work item of the accept pass
                                     (0 = default min(64, max(8, n/4))); autotuned */
    int32_t refresh;              /* lru_refresh */
} lru_config;

/* One operand of a proposal: kmax vector slots per walker (see Conventions).
 * Slot a is one-hot e_{idx[w*kmax + a]} when bit a of onehot_mask is set
 * (the one-hot representation of Sec. 2.2 / 3.2), else dense from `dense`.
 * Mixed operands (e.g. the simultaneous row-and-column update of Sec. 2.2)
 * set some bits.  `dense` may be NULL when every slot is one-hot, `idx` may
 * be NULL when none is. */
typedef struct {
    const void* dense;
    const int32_t* idx;
    uint32_t onehot_mask;
} lru_operand;

typedef struct lru_ctx* lru_handle;

/* ---- life cycle ---------------------------------------------------------- */

/* Validates cfg, allocates the per-walker state on cfg->device (A^{-1} or
 * A_0^{-1}, delay slots, log-value, sign/phase, proposal scratch).  The state
 * stays uninitialised until lru_init_det / lru_init_pf. */
lru_status lru_create(const lru_config* cfg, lru_handle* out);
lru_status lru_destroy(lru_handle h);
/* stream: a cudaStream_t (NULL = legacy default stream). */
lru_status lru_set_stream(lru_handle h, void* stream);
/* bytes of device memory the handle holds */
lru_status lru_device_bytes(lru_handle h, size_t* bytes);

/* ---- initialisation and refresh (Sec. 2.3 init_det_carrier, Sec. 3.3
 *      init_pf_carrier, App. A.1 slogpf) -------------------------------- */

/* A: W matrices (row-major).  Computes A^{-1} by Gauss-Jordan elimination
 * with partial pivoting in FP64 (complex128 for complex dtypes), log|det A|
 * and sign/phase; empties the delay slots.  logabs (W doubles) and sign (W
 * scalars) may be NULL.  Walkers whose A is singular get logabs = -inf,
 * sign = 0 and an unusable inverse. */
lru_status lru_init_det(lru_handle h, const void* A, double* logabs, void* sign);
/* A: W skew-symmetric matrices of even size.  pf by Parlett-Reid skew
 * elimination with pivoting, inverse by Gauss-Jordan, made exactly skew. */
lru_status lru_init_pf(lru_handle h, const void* A, double* logabs, void* sign);
/* Same as init for the walkers with mask[w] != 0 (mask NULL = all).
 * drift (W doubles, may be NULL) receives, per refreshed walker,
 * ||A_tracked^{-1} - A_fresh^{-1}||_F / ||A_fresh^{-1}||_F; log-value and
 * sign are recomputed.  A is the caller's current matrix (the caller owns the
 * configuration, as in the listings of Sec. 2.3 and 3.3). */
lru_status lru_refresh_from_scratch(lru_handle h, const void* A, const uint8_t* mask, double* drift);

/* ---- proposal and acceptance --------------------------------------------- */

/* Determinant proposal (Sec. 2.1; delayed: Sec. 2.3, R_tau equation).
 * ratio (W scalars) = det R; st (W int32, may be NULL) = per-walker status.
 * The proposal is kept until the next propose; U and V must stay valid until
 * lru_accept returns (the accept pass reads V). */
lru_status lru_propose_det(lru_handle h, const lru_operand* U, const lru_operand* V,
                           void* ratio, int32_t* st);
/* Pfaffian proposal (Sec. 3.1 / App. A.2; delayed: Sec. 3.3).  C: W matrices
 * of size 2k x 2k (skew, invertible), or NULL for C = -J (the paper's form,
 * A' = A - B J B^T).  Walker w's C starts at element w * (2 kmax)^2 and is
 * stored row-major as 2k_w x 2k_w (with uniform k: W consecutive 2k x 2k
 * matrices).  ratio = pf(C^{-1} + B^T A^{-1} B) / pf(C^{-1}). */
lru_status lru_propose_pf(lru_handle h, const lru_operand* B, const void* C,
                          void* ratio, int32_t* st);
/* Applies the last proposal to the walkers with mask[w] != 0 (NULL = all)
 * whose proposal status is OK: updates A^{-1} (plain: Eq. det_inv / Woodbury)
 * or stores the new delay slot (Sec. 2.3 / 3.3), adds log|ratio| to log|value|
 * and multiplies the sign/phase.  A walker whose delay slots are full is
 * folded into A_0^{-1} at once (the flush of Eq. delayed_Ainv). */
lru_status lru_accept(lru_handle h, const uint8_t* mask);
/* One persistent fused step for all walkers, including walkers of uneven n
 * and k: a single kernel launch of a fixed grid takes the proposals of every
 * walker (largest first) and then, unless accept == 0, the accept passes, from
 * a device work queue, with bounded waits between a walker's propose and its
 * accept pass.  Acceptance: walkers whose proposal status is OK and, when
 * given, mask[w] != 0 and |ratio|^2 >= u[w] (u: W doubles, Metropolis
 * uniforms).  acc_out (W uint8, may be NULL) receives the decisions.  Plain
 * and delayed handles: in the delayed form (Sec. 2.3 / 3.3) the accept pass
 * stores the walker's new slot and advances its own delay counter tau, and
 * the same launch folds the slots of every walker whose tau reached K into
 * A_0^{-1} (Eqs. delayed_Ainv, pf_delayed_Ainv) in FP64 / complex128 tiles,
 * whatever the handle's flush precision, and resets its tau; walkers with
 * fewer accepted moves keep their slots.  The call issues only a memset and
 * one kernel on the handle's stream (no allocation, no synchronisation), so it can be captured
 * in a CUDA graph; make one call before capturing so that one-time kernel
 * set-up happens outside the capture.  ratio/st as in lru_propose_det; U, V
 * (det) or B (pf, with C or NULL) as in the propose calls. */
lru_status lru_step_persistent(lru_handle h, const lru_operand* U, const lru_operand* V, const void* C,
                               int32_t accept, const uint8_t* mask, const double* u, void* ratio, int32_t* st,
                               uint8_t* acc_out);
/* Folds the partial delay slots of the masked walkers into A_0^{-1} now. */
lru_status lru_flush_delayed(lru_handle h, const uint8_t* mask);

/* ---- state access ------------------------------------------------------- */

/* out: W matrices, row-major, the current A^{-1} (A_0^{-1} with the delayed
 * corrections applied; the state is not changed). */
lru_status lru_get_inverse(lru_handle h, void* out);
/* logabs: W doubles; sign: W scalars (either may be NULL). */
lru_status lru_get_logvalue(lru_handle h, double* logabs, void* sign);
/* tau: W int32, the number of filled delay slots per walker. */
lru_status lru_get_delay(lru_handle h, int32_t* tau);
/* Checkpoint: the whole per-walker state as one opaque device blob. */
lru_status lru_state_bytes(lru_handle h, size_t* bytes);
lru_status lru_save_state(lru_handle h, void* buf);
lru_status lru_load_state(lru_handle h, const void* buf);
/* Synchronises the stream and reports (then clears) the sticky device error. */
lru_status lru_check_device_error(lru_handle h);
/* Self-test of failure detection without a GPU fault: enqueues one warp that
 * waits, with the persistent step's bounded acquire wait, on a device flag
 * that no kernel sets.  After `polls` polls (0 .. 2^24, about 64 ns apart)
 * the wait gives up and sets the sticky LRU_ERR_TIMEOUT, which the next
 * lru_check_device_error returns (and clears); the handle stays usable.
 * LRU_ERR_ARG for polls outside that range. */
lru_status lru_wait_selftest(lru_handle h, int64_t polls);

/* ---- reverse-mode differentiation (adjoint kernels) ----------------------- */

/* log of the pending proposal's ratios into logr (W scalars): log|r| for real
 * dtypes, the principal complex log for complex ones. */
lru_status lru_log_ratio(lru_handle h, void* logr);
/* Vector-Jacobian product of the pending determinant proposal's log ratio
 * (Sec. 2.1, Eqs. det_R, det_ratio): g (W scalars) = dL/dlog r.  Writes
 * gU = g (R^{-1} V A^{-1})^T and gV = g (A^{-1} U R^{-1})^T (operand vector
 * layout, kmax slots; one-hot slots get the dense gradient too) and
 * gA = -g (A^{-1} U R^{-1} V A^{-1})^T (W matrices, row-major).  Complex
 * dtypes return g * conj(J) (the convention of PyTorch's autograd).  Any
 * output may be NULL.  Call after propose and before accept; walkers whose
 * proposal status is not OK get zeros.  The delayed state recomputes V A^{-1}
 * from A_0^{-1} and the stored slots instead of storing A^{-1}. */
lru_status lru_backward_det(lru_handle h, const void* g, void* gU, void* gV, void* gA);
/* Same for the Pfaffian proposal (App. A.2 Eq. pf_low_rank, App. A.3 Eq.
 * pf_grad), with A and C entering through their skew parts (M - M^T)/2:
 * gB = g X M^{-1} (X = A^{-1} B), gA_ij = g (X M^{-1} X^T)_ji / 2, gC = skew
 * part of -g [C^{-1} (M^{-1} - C) C^{-1}]^T / 2 (W x 2k x 2k). */
lru_status lru_backward_pf(lru_handle h, const void* g, void* gB, void* gC, void* gA);
/* d log|det A| / dA = A^{-T} (det) or d log pf A / dA_ij = (A^{-1})_ji / 2 (pf,
 * App. A.3 Eq. pf_grad divided by pf), times g (W scalars): gA row-major. */
lru_status lru_backward_logvalue(lru_handle h, const void* g, void* gA);
/* gPhi[rows[w][i]][:] += gA[w][i][:] for all walkers (rows: W x n int32 into
 * the m x n matrix gPhi): the gradient of the orbital matrix Phi through
 * A_w = Phi[rows_w].  Atomic adds; gPhi is accumulated, not cleared. */
lru_status lru_scatter_rows_add(lru_handle h, const void* gA, const int32_t* rows, int32_t m, void* gPhi);

/* ---- operand formation for QMC moves (Sec. 2.2, 3.2) --------------------- */

/* Determinant row replacement (Sec. 2.2, Eq. det_rank1_row; k > 1: k rows at
 * once, e.g. two-electron moves): walker w moves slot i_a = slot[w*k + a]
 * from orbital row occ[w][i_a] to row new_row[w*k + a] of Phi (m x n
 * row-major, shared by all walkers), a < k.  Writes V_out (vector layout,
 * kmax = k) with row a = Phi[new_a] - Phi[occ_{i_a}] and idx_out[w*k + a] =
 * i_a, so U = [e_{i_a}] (one-hot) and V = V_out (dense).  Slots and new rows
 * of one walker must be distinct.  occ is W x n int32 and is not changed.
 * Uniform-n handles only. */
lru_status lru_form_row_moves(lru_handle h, const void* Phi, int32_t m, const int32_t* occ,
                              const int32_t* slot, const int32_t* new_row,
                              void* V_out, int32_t* idx_out);
/* Pfaffian row-and-column replacement (Eq. pf_rank2): particle i = slot[w]
 * moves from site pos[w][i] to new_site[w]; F is the m x m skew pairing
 * matrix.  Writes B (kmax = 2 vector layout): column 0 = x with
 * x_j = F(r', r_j) - F(r_i, r_j), column 1 one-hot e_i (idx_out[2w+1] = i,
 * idx_out[2w] unused); C = -J.  Handles with k = 2 move two particles at
 * once (Sec. 3.2, the update of 2 rows and 2 columns): slot and new_site are
 * W x 2 (distinct slots p, q; distinct unoccupied sites), B = [x, y, e_p, e_q]
 * (kmax = 4; idx_out[4w+2] = p, idx_out[4w+3] = q, onehot_mask 0b1100) with
 * x_j = F(r'_p, r'_j) - F(r_p, r_j) over the new sites of both particles,
 * y_j = F(r'_q, r_j) - F(r_q, r_j), y_p = 0; C = -J.  Uniform n and k only. */
lru_status lru_form_pf_moves(lru_handle h, const void* F, int32_t m, const int32_t* pos,
                             const int32_t* slot, const int32_t* new_site,
                             void* B_out, int32_t* idx_out);
/* After an accept: occ[w][slot[w*k + a]] = new_row[w*k + a] (a < k; k = 1 for
 * Pfaffian handles) for masked walkers whose proposal was accepted (mask
 * NULL = all). */
lru_status lru_commit_moves(lru_handle h, int32_t* occ, const int32_t* slot,
                            const int32_t* new_row, const uint8_t* mask);

/* Slater matrices for init / refresh: A_w[i][:] = Phi[occ[w][i]][:] (W x n x n,
 * row-major).  Out-of-range rows give zero rows and set the sticky error. */
lru_status lru_gather_rows(lru_handle h, const void* Phi, int32_t m, const int32_t* occ, void* A_out);
/* Pfaffian matrices: A_w[i][j] = F[pos[w][i]][pos[w][j]] (F m x m skew). */
lru_status lru_gather_pairs(lru_handle h, const void* F, int32_t m, const int32_t* pos, void* A_out);

/* ---- standalone batched dense operations (App. A.1) ---------------------- */

/* slogdet of W matrices of size n (row-major), dtype as given. */
lru_status lru_slogdet_batched(int32_t dtype, int64_t W, int32_t n, const void* A,
                               double* logabs, void* sign, void* stream);
/* Same as lru_slogdet_batched, but allocates nothing (the paper has no
 * counterpart; this is a deployment variant).  For callers that cannot let a
 * library allocate device memory: runtimes that reserve most of the GPU for
 * their own memory pool, code that must avoid the device-wide synchronisation
 * of cudaFree, and code recorded once and replayed later.  The Gauss-Jordan
 * workspace is a fixed 64 MiB array in the library's device memory, which
 * every GPU that loads the library holds until the process exits.  Limit:
 * one n x n matrix must fit it (n * n * sizeof(scalar) <= 64 MiB, so every
 * n <= 2048 of every dtype); other sizes return LRU_ERR_ARG.  The first call on a
 * device looks up the workspace's address for that device (a runtime query,
 * no allocation): make that first call before any stream capture.  All calls
 * share the one workspace, whose contents persist between calls; every matrix
 * is copied in before use, so nothing needs clearing, but calls whose work
 * overlaps on the GPU (different streams or host threads without ordering)
 * race on it and must be serialised by the caller. */
lru_status lru_slogdet_batched_noalloc(int32_t dtype, int64_t W, int32_t n, const void* A,
                                       double* logabs, void* sign, void* stream);
/* slogpf of W skew matrices of even size n (Parlett-Reid with pivoting). */
lru_status lru_slogpf_batched(int32_t dtype, int64_t W, int32_t n, const void* A,
                              double* logabs, void* sign, void* stream);
/* Vector-Jacobian products of the two calls above (App. A.3, Eq. pf_grad; for
 * the determinant the classical d log det A = tr(A^{-1} dA)).  Inputs: the same
 * A (W row-major n x n), g_logabs (W doubles, dL/dlog|value|, or NULL = 0),
 * g_sign (W scalars, dL/dsign in torch's convention for complex, or NULL; real
 * signs are piecewise constant and get no gradient) and sign (the forward's
 * sign / phase output, needed when g_sign is given).  Output gA (W row-major
 * n x n, caller-owned): with c = g_logabs + i beta, beta = -Im(conj(g_sign) sign),
 * gA = c A^{-H} (determinant; real: g_logabs A^{-T}) or (c / 2) times the
 * conjugate transpose of the skew part of A^{-1} (Pfaffian: the gradient with
 * respect to A through its skew projection).  The inverses are formed in FP64
 * / complex128 (Gauss-Jordan) in a workspace allocated on the stream for the
 * call.  A singular A gives non-finite gradients.  W <= INT32_MAX, n <= 2048,
 * n even for the Pfaffian. */
lru_status lru_slogdet_backward(int32_t dtype, int64_t W, int32_t n, const void* A, const double* g_logabs,
                                const void* g_sign, const void* sign, void* gA, void* stream);
lru_status lru_slogpf_backward(int32_t dtype, int64_t W, int32_t n, const void* A, const double* g_logabs,
                               const void* g_sign, const void* sign, void* gA, void* stream);

/* ---- profiling (CUDA events on the handle's stream) ----------------------- */

/* Kernel classes timed when profiling is on. */
#define LRU_PROF_PROPOSE 0   /* the propose kernel(s) */
#define LRU_PROF_ACCEPT 1    /* the accept pass over A^{-1} (the Woodbury / GEMV pass) */
#define LRU_PROF_FLUSH 2     /* the delayed flush contraction */
#define LRU_PROF_REFRESH 3   /* from-scratch inverse (and Pfaffian) */
#define LRU_PROF_REFRESH_PANEL 4    /* within REFRESH (tensor-core form): the FP64 panel eliminations */
#define LRU_PROF_REFRESH_UPDATE 5   /* within REFRESH (tensor-core form): the split-product trailing updates */
#define LRU_PROF_CLASSES 6
/* on != 0: record a CUDA event pair around every launch of each class. */
lru_status lru_profile_enable(lru_handle h, int32_t on);
/* Synchronises the stream; total_ms / launches (either may be NULL) receive
 * the summed event time and the number of timed launches of class cls since
 * the last read, which resets them. */
lru_status lru_profile_read(lru_handle h, int32_t cls, double* total_ms, int64_t* launches);
/* Number of kernels this handle has launched (all classes), since creation. */
lru_status lru_launch_count(lru_handle h, int64_t* count);

const char* lru_status_string(lru_status s);
/* "lrugb <version> sm_103a" */
const char* lru_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LRUGB_H */
