// Internal interface between the C-ABI (lrugb_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lru {

// Per-walker geometry, as seen by kernels.  Walker w has an n_w x n_w
// inverse starting at element moff(w) (sum of n_v^2 before it) and length-n_w
// vectors starting at voff(w) (sum of n_v before it) times the slot count.
struct DevLayout {
    int W;
    int n_uni;                 // > 0: every walker has this n (moff, voff computed)
    int n_max;                 // largest n (workspace slot size n_max^2)
    const int* n;              // per-walker n (ragged)
    const long long* moff;
    const long long* voff;
    int kk;                    // vector slots per update (det: k, pf: 2k), max over walkers
    const int* kvec;           // per-walker vector count, or nullptr (= kk)
    int Kc;                    // delay columns per walker row of P, Q (K * kk), 0 if plain
    int K;                     // delay length (>= 2 for the delayed form)
    int Kc32;                  // row stride (elements) of the split copies: Kc rounded up to 32 (TF32) or 64 (BF16)
    long long rows;            // sum of n over walkers (rows of P, Q)
    __device__ __forceinline__ int nw(int w) const { return n_uni > 0 ? n_uni : n[w]; }
    __device__ __forceinline__ long long mo(int w) const {
        return n_uni > 0 ? (long long)w * n_uni * n_uni : moff[w];
    }
    __device__ __forceinline__ long long vo(int w) const {
        return n_uni > 0 ? (long long)w * n_uni : voff[w];
    }
    __device__ __forceinline__ int kv(int w) const { return kvec ? kvec[w] : kk; }
};

// Per-walker state and proposal scratch (one device allocation).
template <typename T>
struct DevState {
    T* G;          // A^{-1} (plain) or A_0^{-1} (delayed), column-major per walker
    T* P;          // delayed: n_w x Kc per walker, row j contiguous
    T* Q;
    int split_bf16;  // 0: the split copies are TF32 in fp32 words; 1: bf16
    float* P32h;   // delayed, tensor-core flush: split copies of P and Q (K-major rows of Kc32)
    float* P32l;
    float* Q32h;
    float* Q32l;
    int* tau;      // filled delay slots per walker
    double* logabs;
    T* sgn;        // sign (real) or unit phase (complex)
    // scratch of the last proposal
    T* X;          // A^{-1} U (det) or A^{-1} B (pf): kk vectors of n_w
    T* Rinv;       // kk x kk per walker: R^{-1} (det) or M^{-1} (pf)
    T* ratio;      // W
    int* pst;      // W proposal status
    T* VP;         // det delayed: V P (MAXKK x Kc per walker)
    T* QtU;        // delayed, dense U columns: Q^T U (Kc x MAXKK per walker)
    int* err;      // sticky device error word
};

struct DevOperand {
    const void* dense;
    const int* idx;
    unsigned mask;   // bit a: slot a is one-hot
    int slots;       // vector slots per walker in the buffers (kmax)
    int pre = -1;    // dense slot whose A^{-1} u_a a separate pass has already written to X (-1: none)
};

// Control block of the persistent fused step (see k_step).
struct StepCtl {
    int* counter;             // work-queue head, zeroed before each launch
    int* prop_done;           // W flags, zeroed before each launch
    int* items_done;          // W counters, zeroed before each launch
    int* fin;                 // W flags: the walker's propose, accept and commit are done (zeroed)
    int* flush_done;          // W counters of finished flush strips (zeroed)
    uint8_t* acc;             // W accept decisions (output)
    const int* order;         // W walkers in propose order
    const int4* acc_items;    // accept items (walker, l0, l1, use_smem), largest walkers first
    const int* nacc_w;        // accept items per walker
    int nacc;
    const int2* flush_items;  // delayed form: flush strips (walker, 32-column block), largest walkers first
    const int* nflush_w;      // flush strips per walker
    int nflush;
    int do_accept;            // 0: propose only
    const uint8_t* mask;      // optional acceptance mask
    const double* u;          // optional Metropolis uniforms: accept if |r|^2 >= u
};

// ---- launchers (defined in lru_kernels.cu, instantiated for every dtype) ----
// df: the pass over A^{-1} for a single dense column in double-float arithmetic (F64 only)
template <typename T>
void launch_propose(bool pf, bool delayed, bool df, const DevLayout& L, const DevState<T>& S, const DevOperand& U,
                    const DevOperand& V, const T* C, T* ratio_out, int* st_out, cudaStream_t st);
template <typename T>
// df: the delayed rank-1 determinant GEMV in double-float arithmetic (F64 only)
void launch_accept(bool pf, bool delayed, bool df, const DevLayout& L, const DevState<T>& S, const DevOperand& V,
                   const uint8_t* mask, const int* items, int nitems, cudaStream_t st);
template <typename T>
void launch_flush_native(bool pf, const DevLayout& L, const DevState<T>& S, const uint8_t* force_mask,
                         int nwalkers_tiles, cudaStream_t st);
void launch_flush_df(bool pf, const DevLayout& L, const DevState<double>& S, const uint8_t* force_mask,
                     cudaStream_t st);
template <typename T>
void launch_flush_finish(const DevLayout& L, const DevState<T>& S, const uint8_t* force_mask, cudaStream_t st);
template <typename T>
void launch_get_inverse(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, T* out, cudaStream_t st);
template <typename T>
void launch_form_row_moves(const DevLayout& L, const T* Phi, int m, const int* occ, const int* slot,
                           const int* newrow, T* Vout, int* idx, cudaStream_t st);
template <typename T>
void launch_form_pf_moves(const DevLayout& L, const T* F, int m, const int* pos, const int* slot,
                          const int* newsite, T* Bout, int* idx, cudaStream_t st);
template <typename T>
void launch_gather(bool pairs, const DevLayout& L, const T* src, int m, const int* occ, T* A, int* err,
                   cudaStream_t st);
template <typename T>
void launch_step(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const DevOperand& U,
                 const DevOperand& V, const T* C, T* ratio_out, int* st_out, const StepCtl& ctl, int grid,
                 cudaStream_t st);
template <typename T>
void launch_zero_split_tail(const DevLayout& L, const DevState<T>& S, const uint8_t* force, cudaStream_t st);
// ---- refresh with the trailing updates on the tensor cores (refresh_oz.cu) ----
constexpr int OZ_B = 64;   // panel width = inner dimension of each trailing update
constexpr int OZ_S = 7;    // BF16 slices per operand (8 bits each: 56 bits)
struct OzWork {
    double* M;        // W x n x n row-major working matrix (M = A^T, inverted in place)
    int* perm;        // W x n pivot rows
    double* logacc;   // W running log|det|
    double* sgnacc;   // W running sign
    int* sing;        // W zero-pivot flags
    uint16_t* Sb;     // W x OZ_S x n x OZ_B  BF16 slices of the columns of S (panel rows of M)
    uint16_t* Pb;     // W x OZ_S x n x OZ_B  BF16 slices of the rows of (panel - E)
    int* eS;          // W x n  power-of-two exponents of the S columns
    int* eP;          // W x n  power-of-two exponents of the panel rows
    uint8_t* go;      // W      walkers that flush now (split-product flush)
    int* cs;          // W x 64 exponent shifts of the slot columns (split-product flush)
    double* piv;      // W x n  pivots of the register panel kernel (log|det| and sign at the end)
};
// columns a split-product update writes: [c_lo, c_hi) minus [s_lo, s_hi), in
// the 128-column tiles jt_lo .. jt_hi - 1
struct OzCols {
    int c_lo, c_hi, s_lo, s_hi, jt_lo, jt_hi;
};
size_t oz_work_bytes(int W, int n);
void oz_work_carve(OzWork& Z, void* base, int W, int n);
void launch_oz_load(int W, int n, const double* A, double* M, const uint8_t* mask, cudaStream_t st);
void launch_oz_panel(int W, int w0, int n, int k0, const OzWork& Z, const uint8_t* mask, cudaStream_t st);
// one 16-column sub-panel (n <= 1024): elimination and its row exchanges on the
// other panel columns; the last one of a panel also exchanges the outside columns
// the tensor-core refresh eliminates its panels in FP64 sub-panels (pivots
// recorded per row, log|det| summed at the end) up to this n
constexpr int OZ_SUBPANEL_MAX_N = 2048;
// width of the FP64 sub-panels of the tensor-core refresh for this n (16, or 8
// above n = 1024, where a thread holds four rows)
int oz_subpanel_width(int n);
bool launch_oz_subpanel(int W, int n, int k0, int sp, const OzWork& Z, const uint8_t* mask, cudaStream_t st);
void launch_oz_finish(int W, int n, const OzWork& Z, const DevState<double>& S, const uint8_t* mask, bool delayed,
                      bool reset_tau, cudaStream_t st);
void launch_oz_drift_store(int W, int n, const DevLayout& L, const DevState<double>& S, const double* M,
                           const uint8_t* mask, double* drift, bool delayed, cudaStream_t st);
// delayed flush A_0^{-1} += sgnQ * P Q^T (determinant: -1, Pfaffian: +1) as the
// same exact split product (uniform n, n % 128 == 0, Kc <= 64); walkers with
// tau >= K, or force && tau > 0 (their go flags stay set for launch_skew_project)
bool launch_flush_split(int W, int n, int K, int Kc, int kk, const double* P, const double* Q, double sgnQ,
                        const int* tau, const uint8_t* force, const OzWork& Z, int* err, cudaStream_t st);
// A_0^{-1} of the walkers with go[w] set: the lower triangle := the exact
// negative of the upper, diagonal 0 (after the Pfaffian split-product flush; n % 32 == 0)
void launch_skew_project(int W, int n, double* G, const uint8_t* go, cudaStream_t st);
// hook(ctx, class, begin) brackets the panel (class 4) and update (class 5) launches
bool launch_refresh_oz(int W, int n, const double* A, const OzWork& Z, const DevState<double>& S,
                       const uint8_t* mask, bool delayed, bool reset_tau, int* err, cudaStream_t st,
                       void (*hook)(void*, int, int), void* hctx);
void launch_wait_selftest(const int* flag, long long iters, int* err, cudaStream_t st);
void launch_commit_moves(int W, int n, int k, int* occ, const int* slot, const int* newrow, const uint8_t* mask,
                         const int* pst, cudaStream_t st);
template <typename T>
void launch_set_delay_zero(const DevLayout& L, const DevState<T>& S, cudaStream_t st);

// ---- refresh / dense (refresh.cu) ----
// For each selected walker: G := A^{-1} (column-major) by Gauss-Jordan on A^T,
// log|det| and sign into S (write_logdet), tau := 0.  With ws (nws slots of
// n_uni^2 scalars) the inverse is formed in the CTA's slot first and the drift
// of the tracked inverse against it is written before it replaces G.
template <typename T>
void launch_refresh(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const T* A,
                    const uint8_t* mask, T* ws, int nws, double* drift, bool write_logdet, cudaStream_t st);
// Pfaffian (Parlett-Reid) of the selected walkers' A into logabs / sgn; ws: nws slots.
template <typename T>
void launch_slogpf(const DevLayout& L, const T* A, const uint8_t* mask, T* ws, int nws, double* logabs, T* sgn,
                   cudaStream_t st);
template <typename T>
void launch_slogdet(int W, int n, const T* A, T* ws, int nws, double* logabs, T* sgn, cudaStream_t st);

// ---- adjoint (adjoint.cu) ----
template <typename T>
void launch_backward(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const DevOperand& V,
                     const T* C, const T* g, T* ws, T* gU, T* gV, T* gA, T* gC, cudaStream_t st);
template <typename T>
void launch_backward_logvalue(bool pf, bool delayed, const DevLayout& L, const DevState<T>& S, const T* g, T* gA,
                              cudaStream_t st);
template <typename T>
void launch_log_ratio(int W, const T* ratio, T* out, cudaStream_t st);
// gradient of (sign, log|det|) or (phase, log|pf|) from the column-major inverses
template <typename T>
void launch_slog_grad(int W, int n, bool pf, const T* Ginv, const double* g_l, const T* g_s, const T* sign, T* gA,
                      cudaStream_t st);
template <typename T>
void launch_scatter_rows(const DevLayout& L, const T* gA, const int* rows, int m, T* gPhi, int* err, cudaStream_t st);

// ---- tensor-core flush (flush_tc.cu) ----
// Returns false when the combination is not built.
bool launch_flush_tc(int mode, bool pf, const DevLayout& L, double* G, const void* Ph, const void* Pl,
                     const void* Qh, const void* Ql, const int* tau, const uint8_t* force_mask,
                     int* err, cudaStream_t st);

}  // namespace lru
