/*
 * cc3.h -- C ABI of the GB300 CC3 triples library (libcc3.so).
 *
 * The library computes the closed-shell CC3 triples contribution to the
 * coupled-cluster residual and to the right Jacobian transformation, following
 * Paul, Myhre and Koch, "A new and efficient implementation of CC3"
 * (arXiv 2007.01088), section "Implementation", Algorithms 1 and 2 and
 * eq. "jcc3".  Everything runs in CUDA kernels on one GPU (sm_103a).
 *
 * Index conventions (row-major, float64, indices in the order written):
 *   no occupied (active) and nv virtual orbitals
 *   eps_o[no], eps_v[nv]                orbital energies (Eh)
 *   t2[i][j][a][b]  = t^{ab}_{ij}        doubles amplitudes
 *   g_vvvo[b][d][c][k] = (bd|ck)         two-electron integrals (chemists'
 *   g_ooov[l][j][k][c] = (lj|kc)         notation, real orbitals, full 8-fold
 *   g_ovov[j][b][k][c] = (jb|kc)         permutational symmetry, T1 = 0)
 *   F_ov[k][c]                           occupied-virtual Fock block
 *   chol_L[J][p][q]                      Cholesky vectors over the no+nv
 *                                        orbitals (occupied first), optional
 *   R1[n][i][a], R2[n][i][j][a][b]       trial vectors
 *   Omega1[i][a], Omega2[i][j][a][b], rho1[n][i][a], rho2[n][i][j][a][b]
 *
 * Ownership: the caller owns every buffer it passes.  cc3_ctx_create copies
 * its inputs into device memory owned by the context (device-to-device with
 * CC3_DEVICE_PTRS); the context frees them in cc3_ctx_destroy.  Outputs are
 * overwritten with the triples contribution only (the caller adds it to its
 * CCSD residual).  With CC3_DEVICE_PTRS every pointer argument of every call
 * on that context (inputs and outputs) is a device pointer; otherwise all are
 * host pointers and the call copies and synchronises.
 *
 * Threading: calls on one context are serialised by the caller; distinct
 * contexts may be used from different threads.  cuda_stream may be NULL (the
 * legacy default stream) or a cudaStream_t.
 *
 * Errors: every call returns a status (CC3_OK = 0, negative on error) and
 * never aborts the process; cc3_strerror names it.  A device-side failure is
 * reported through a device status word and surfaces as CC3_ERR_TIMEOUT or
 * CC3_ERR_CUDA.
 */
#ifndef CC3_H
#define CC3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc3_ctx cc3_ctx;
typedef struct cc3_server cc3_server;

/* Arithmetic of the bulk contractions.
 * CC3_FP64       native FP64 everywhere: the contractions run as FP64 fused
 *                multiply-adds on the FP64 pipe (DFMA), the element-wise
 *                steps and all sums in FP64.
 * CC3_SPLIT_BF16 the dominant contractions run as exact products of
 *                integer-valued BF16 slices of the FP64 operands on the
 *                tensor cores (FP32 accumulation of exact integer sums),
 *                recombined in extended precision.  The denominators and
 *                the contravariant combination run in double-float
 *                arithmetic (pairs of FP32, ~48 significant bits); the
 *                cross-triple accumulation and the energy stay in FP64.
 * CC3_SPLIT_INT8 reserved (the INT8 tensor rate of this GPU is far below its
 *                BF16 rate); returns CC3_ERR_UNSUPPORTED. */
typedef enum { CC3_FP64 = 0, CC3_SPLIT_BF16 = 1, CC3_SPLIT_INT8 = 2 } cc3_prec;

enum {
  CC3_OK = 0,
  CC3_ERR_ARG = -1,         /* invalid argument (size, pointer, flag)        */
  CC3_ERR_OOM = -2,         /* device or host allocation failed               */
  CC3_ERR_CUDA = -3,        /* a CUDA call or kernel launch failed            */
  CC3_ERR_TIMEOUT = -4,     /* a bounded device wait gave up                  */
  CC3_ERR_DENOM = -5,       /* |w - eps| < CC3_DENOM_MIN or eps <= 0 somewhere */
  CC3_ERR_BUSY = -6,        /* server full / request rejected at admission    */
  CC3_ERR_UNSUPPORTED = -7, /* option not available in this build             */
  CC3_ERR_NOT_FOUND = -8,   /* unknown ticket                                  */
  CC3_ERR_CANCELLED = -9    /* request cancelled / server stopped              */
};

/* Smallest distance |w - eps^{abc}_{ijk}| (Eh) between a Jacobian frequency
 * and a triples denominator that cc3_jacobian_triples accepts: closer, the
 * R3 amplitudes (w - eps)^{-1} <mu3|...> sit on a pole of the effective
 * Jacobian and the call returns CC3_ERR_DENOM instead. */
#define CC3_DENOM_MIN 1e-6

/* flags of cc3_ctx_create */
#define CC3_DEVICE_PTRS 1u   /* all pointers of this context are device pointers */
#define CC3_DETERMINISTIC 2u /* order-independent cross-triple sums of the     */
                             /* residual (128-bit fixed-point accumulation with */
                             /* integer atomics, 2^-64 resolution): bitwise     */
                             /* reproducible Omega1/Omega2/E_T on both paths.   */
                             /* cc3_jacobian_triples then returns               */
                             /* CC3_ERR_UNSUPPORTED.  Without it the sums use   */
                             /* FP64 atomics (reproducible to rounding).        */

/* Create a context for one problem (no >= 1, 1 <= nv <= 1024).  Uploads and
 * reorders the inputs (paper: integrals are reordered before the triple loop,
 * "Implementation" section).  chol_L may be NULL (naux = 0): then the
 * Jacobian is unavailable (CC3_ERR_ARG).  Returns CC3_ERR_DENOM when some
 * ground-state denominator eps^{abc}_{ijk} = e_a + e_b + e_c - e_i - e_j - e_k
 * could be <= 0 (3 min eps_v <= 3 max eps_o).  On success *out owns device
 * memory of about (5 nv^3 no + 4 no^2 nv^2) * 8 bytes plus per-call workspace. */
int cc3_ctx_create(cc3_ctx **out, int no, int nv, const double *eps_o,
                   const double *eps_v, const double *t2, const double *g_vvvo,
                   const double *g_ooov, const double *g_ovov,
                   const double *F_ov, const double *chol_L, int naux,
                   unsigned flags, void *cuda_stream);

/* Context for general integrals, as the T1-transformed Hamiltonian of a CC3
 * iteration with t1 != 0 gives them (paper, "Implementation": the integrals
 * are T1 transformed and lose the pq <-> qp symmetry, so no block can be
 * derived from another).  The five blocks of Algorithm 1 come separately:
 *   g_vvvo[b][d][c][k] = g_bdck      g_oovo[l][j][c][k] = g_ljck
 *   g_ooov[j][l][k][c] = g_jlkc      g_ovov[j][b][k][c] = g_jbkc
 *   g_vvov[d][b][k][c] = g_dbkc      F_ov[k][c] (the T1-transformed Fock block)
 * The W build reads vvvo and oovo, the contractions vvov, ooov, ovov and F
 * (for symmetric integrals g_oovo is g_ooov with its last two indices swapped
 * and g_vvov[d][b][k][c] = g_vvvo[b][d][c][k], which is what cc3_ctx_create
 * assumes).  eps_o and eps_v are the orbital energies of the denominators.
 * Other arguments, ownership and errors as cc3_ctx_create; the residual
 * (cc3_omega_triples) runs on both precision paths, while
 * cc3_jacobian_triples on such a context returns CC3_ERR_UNSUPPORTED (its
 * R1 dressing assumes symmetric integrals). */
int cc3_ctx_create_general(cc3_ctx **out, int no, int nv, const double *eps_o,
                           const double *eps_v, const double *t2, const double *g_vvvo,
                           const double *g_oovo, const double *g_ooov, const double *g_ovov,
                           const double *g_vvov, const double *F_ov, unsigned flags,
                           void *cuda_stream);

void cc3_ctx_destroy(cc3_ctx *ctx);

/* Restrict the triple loop to ntri unique occupied triples ijk[3*t..3*t+2]
 * with i >= j >= k (host pointer, copied).  ntri = 0 or ijk = NULL restores the
 * full loop (all i >= j >= k, paper Algorithm 1).  The results are then the
 * contributions of exactly those triples (used for sampled checks and for
 * task filters such as core-valence separation). */
int cc3_ctx_set_triples(cc3_ctx *ctx, int ntri, const int *ijk);

/* Core-valence separation task filter (paper, Introduction and
 * Applications: the triple loop skips every occupied triple none of whose
 * indices is a core orbital of interest, which takes the Jacobian from
 * 8 nv^4 no^3 to 8 nv^4 no^2 per vector for one core orbital).  Host only,
 * no context needed.  core[ncore]: distinct occupied indices in [0, no).
 * Enumerates the triples i >= j >= k, not all equal, with at least one index
 * in core, in loop order (i outermost), and writes the first min(count, max)
 * of them to ijk[3 * t + 0..2] (ijk may be NULL when max = 0).  Returns the
 * count (>= 0), or CC3_ERR_ARG for no < 0, ncore < 0 or > no, a NULL core
 * with ncore > 0, an index outside [0, no) or a repeated index.  Pass the
 * result to cc3_ctx_set_triples to restrict a context to those tasks. */
int cc3_cvs_triples(int no, int ncore, const int *core, int max, int *ijk);

/* CC3 triples contribution to the ground-state residual (Algorithm 1):
 * Omega1[no][nv], Omega2[no][no][nv][nv] (covariant, pair symmetric) and
 * E_T = sum_{ijab} t^{ab}_{ij} Omega~^{ab}_{ij} (the contravariant residual
 * paired with the amplitudes).  Any output pointer may be NULL. */
int cc3_omega_triples(cc3_ctx *ctx, cc3_prec prec, double *Omega1,
                      double *Omega2, double *E_T, void *cuda_stream);

/* Right CC3 Jacobian transformation (triples part) of nvec trial vectors at
 * frequencies omega[nvec] (host array always):
 *   R3 = (w - eps)^{-1} <mu3| [H,R2] + [[H,R1],T2] >,
 *   rho = <mu1|[H,R3]> (+) <mu2|[H,R3]> + <mu2|[[H,R1],T3]>   (eq. "jcc3")
 * with H the T1-transformed Hamiltonian; the R1 dressing of the integrals
 * needs the Cholesky vectors.  The tau3-dependent intermediates of
 * Algorithm 2 are built on first use and cached in the context.
 * rho1[nvec][no][nv], rho2[nvec][no][no][nv][nv].  Before any device work the
 * call checks every frequency against the denominators of the context's
 * triple loop (cc3_denominator_gap) and returns CC3_ERR_DENOM if one of them
 * comes within CC3_DENOM_MIN of some eps^{abc}_{ijk} (CC3_ERR_ARG for a
 * non-finite frequency). */
int cc3_jacobian_triples(cc3_ctx *ctx, cc3_prec prec, int nvec,
                         const double *omega, const double *R1,
                         const double *R2, double *rho1, double *rho2,
                         void *cuda_stream);

/* Left (transpose) CC3 Jacobian transformation (triples part) of nvec left
 * vectors at frequencies omega[nvec] (host array always), the product needed
 * for left excited states and for the multipliers (paper, "Implementation",
 * the transpose-Jacobian paragraph; the L3 amplitudes of Algorithm 3):
 *   L3 = (w - eps)^{-1} P[ L1 (x) g_ovov + L2~ (x) F + contractions of L2~ with
 *        g_vvov and g_ooov ],  L2~ = the back-transform applied to L2,
 * then its contravariant form contracted with the integrals (sigma2) and with
 * t2 into intermediates that the Cholesky vectors turn into sigma1, after a
 * loop that contracts tau3 (sharing the Algorithm 2 intermediates with
 * cc3_jacobian_triples).  The result is the exact transpose of the right
 * transformation under the plain inner product over the elements of (R1, R2):
 *   sum L1 . rho1(R) + sum L2 . rho2(R) = sum sigma1(L) . R1 + sum sigma2(L) . R2
 * for every R with pair-symmetric R2; sigma2 is pair symmetric.
 * L1[n][i][a], L2[n][i][j][a][b], sigma1[n][i][a], sigma2[n][i][j][a][b]; other
 * rules (pointers, frequencies, CC3_ERR_DENOM, symmetric integrals, Cholesky
 * vectors required) as cc3_jacobian_triples.  CC3_FP64 or CC3_SPLIT_BF16 (the
 * W build, the contractions of tau3 and L3, the G, H, Q intermediates and the
 * Cholesky product of sigma1 on the tensor cores, the rest of sigma1 in FP64;
 * CC3_SPLIT_INT8 returns CC3_ERR_UNSUPPORTED). */
int cc3_left_jacobian_triples(cc3_ctx *ctx, cc3_prec prec, int nvec, const double *omega,
                              const double *L1, const double *L2, double *sigma1,
                              double *sigma2, void *cuda_stream);

/* Triples contributions to the one-electron density of a left state
 * (paper, "Implementation", Algorithm 3): for the left state (L1, L2) at
 * frequency omega,
 *   D_vv[c][d] =  1/2 sum_{ijkab} L3~^{abc}_{ijk} tau^{abd}_{ijk}
 *   D_oo[l][k] = -1/2 sum_{ijabc} L3~^{abc}_{ijk} tau^{abc}_{ijl}
 *   D_ov[k][c] =  sum_{ijab} L2~^{ab}_{ij} tau~^{abc}_{ijk}
 *                - sum_{cik} Y^o_{clik} t^{cd}_{ki}  (at [l][d]),
 *   Y^o_{clik} = sum_{jab} L3~^{abc}_{ijk} t^{ab}_{lj},
 * with tau = -W / eps (Algorithm 1), L3 the covariant amplitudes of
 * cc3_left_jacobian_triples, L3~ their contravariant form and L2~ the
 * back-transform applied to L2; the vo block has no triples term.  The
 * occupied loop runs over the triples i >= j >= k.  On CC3_FP64 the D_oo term
 * runs over Algorithm 3's virtual loop a >= b >= c; on CC3_SPLIT_BF16 the
 * occupied loop's contractions run on the tensor cores and D_oo comes from tau
 * and L3~ of every triple (i = j = k included) held resident in device memory,
 * 16 nv^3 bytes per triple (CC3_ERR_OOM when that exceeds half of the free
 * memory; the FP64 path has no such limit).  With omega = 0 and the
 * ground-state multipliers in place of (L1, L2) the call gives D^{0,0}.
 * L1[no][nv], L2[no][no][nv][nv] (host, or device with CC3_DEVICE_PTRS);
 * outputs D_oo[no][no], D_ov[no][nv], D_vv[nv][nv], overwritten.  Before any
 * device work: CC3_ERR_ARG for a null pointer or a non-finite omega,
 * CC3_ERR_DENOM if omega comes within CC3_DENOM_MIN of any eps^{abc}_{ijk}
 * (i >= j >= k, i = j = k included: the virtual loop divides there too),
 * CC3_ERR_UNSUPPORTED for a context with general (T1-transformed) integrals,
 * a restricted triples list, deterministic mode, CC3_SPLIT_INT8, or more than
 * 24 occupied orbitals on CC3_FP64.  Cost 10 nv^4 no^3 FLOP to leading order
 * (6 nv^4 per distinct permutation in the occupied loop, 4 nv^4 no^3 in the
 * virtual loop; the counters report this count on both paths). */
int cc3_density_triples(cc3_ctx *ctx, cc3_prec prec, double omega, const double *L1,
                        const double *L2, double *D_oo, double *D_ov, double *D_vv,
                        void *cuda_stream);

/* Smallest |w - eps^{abc}_{ijk}| over every virtual triple (a, b, c) and the
 * occupied triples of a loop, eps^{abc}_{ijk} = e_a + e_b + e_c - e_i - e_j -
 * e_k (the R3 denominator of eq. "jcc3" at frequency w; at w = 0 the tau
 * denominator of Algorithm 1).  Host only, no context needed: eps_o[no],
 * eps_v[nv] are host arrays; ntri = 0 (ijk may be NULL) means the full loop
 * i >= j >= k, not all equal, else ijk[3 t + 0..2] lists the triples
 * (i >= j >= k).  Writes the distance to *gap (1e300 if the loop is empty).
 * CC3_ERR_ARG for sizes < 1, NULL pointers, a triple out of order or out of
 * range, or non-finite energies or frequency. */
int cc3_denominator_gap(int no, int nv, const double *eps_o, const double *eps_v, int ntri,
                        const int *ijk, double w, double *gap);

/* Counters of the last call on ctx: nominal FLOP (4 nv^4 no^3 per residual,
 * 8 nv^4 no^3 per trial vector, over the triples in the loop), FLOP executed
 * by the FP64 or slice products, and the number of kernel launches. */
typedef struct {
  double nominal_flop;
  double executed_flop;
  long long launches;
  int slices;              /* BF16 slices per operand (split path), else 0 */
} cc3_counters;
int cc3_ctx_counters(const cc3_ctx *ctx, cc3_counters *out);

/* FP64 triples residual that allocates no device memory (the paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc, e.g. code
 * embedded in a host application that owns the whole GPU memory pool, or code
 * running while the application forbids new allocations).  Same result as
 * cc3_omega_triples(ctx, CC3_FP64, ...) on the same inputs.  All pointers are
 * DEVICE pointers owned by the caller, with the layouts of cc3_ctx_create and
 * cc3_omega_triples; any output may be NULL.  Every piece of scratch (a
 * transposed integral block, one triple's W and tau~, the residual
 * accumulators, reduction partials and contraction tables) comes from one
 * 16 MiB file-scope device array that every GPU loading the library keeps
 * until process exit; it limits the size to no <= 12, nv <= 64 (larger sizes
 * return CC3_ERR_ARG).  The first call on a device (and the first after that
 * device's context was reset) looks the array's address up for it; make that
 * first call before any stream capture.  Calls share the array: calls that
 * overlap on the GPU race.  Each call reads eps_o and eps_v back to the host
 * and returns CC3_ERR_DENOM, with nothing enqueued, when some denominator
 * could be <= 0 (3 min eps_v <= 3 max eps_o), as cc3_ctx_create does.  It
 * synchronises cuda_stream twice (after reading the orbital energies and after
 * uploading its tables into the array) and returns after enqueuing its kernels
 * on cuda_stream.  Because it reads back and synchronises, the call cannot be
 * recorded into a CUDA graph, and it must not run while another thread
 * captures a stream in cudaStreamCaptureModeGlobal. */
int cc3_omega_triples_noalloc(int no, int nv, const double *eps_o, const double *eps_v,
                              const double *t2, const double *g_vvvo,
                              const double *g_ooov, const double *g_ovov,
                              const double *F_ov, double *Omega1, double *Omega2,
                              double *E_T, void *cuda_stream);

/* Kernel tracing.  With tracing on, every library kernel launch is bracketed
 * by CUDA events recorded on the launching stream, grouped by kernel class;
 * cc3_ctx_trace returns, for the last call, each class's launches, summed
 * device time (ms) and algorithmic FLOP (FP64-equivalent useful FLOP of the
 * contractions; for the split engine also the BF16 slice-product FLOP).
 * Tracing synchronises the stream at the end of each call. */
typedef struct {
  char name[32];
  long long launches;
  double ms;
  double flop;        /* FP64-equivalent useful FLOP                     */
  double slice_flop;  /* BF16 slice-product FLOP (split engine), else 0 */
} cc3_trace_entry;
typedef struct {
  int n;
  cc3_trace_entry e[8];
} cc3_trace;
int cc3_ctx_set_tracing(cc3_ctx *ctx, int on);
int cc3_ctx_trace(const cc3_ctx *ctx, cc3_trace *out);

/* Set the number of BF16 slices per FP64 operand of the split path
 * (3 <= s <= 7; default 6: 48 bits per operand, which keeps the residual
 * within 1e-9 absolute and the energy within 1e-8 Eh at the no = 16,
 * nv = 160 scale).  */
int cc3_ctx_set_slices(cc3_ctx *ctx, int slices);

/* Autotuner of the split path (no counterpart in the paper, whose CPU code
 * has no tile shapes to choose): times the residual on a strided sample of
 * about 32 triples of the context's loop for each candidate tiling (K steps
 * per tile of the vvov contraction: 200, 400, 800; N tile of the W build:
 * the default and the next smaller one), keeps the fastest for this context
 * and for every later context of the same (no, nv, slices) in the process,
 * and returns it (either output pointer may be NULL).  Runs kernels on
 * cuda_stream; the context's Omega accumulators are scratch meanwhile. */
int cc3_ctx_autotune(cc3_ctx *ctx, void *cuda_stream, int *ksteps_per_tile, int *ntile_w);
/* The split path's current tiling (tuned or default). */
int cc3_ctx_get_tuning(cc3_ctx *ctx, int *ksteps_per_tile, int *ntile_w);

const char *cc3_strerror(int status);

/* Detail of the most recent failure on the calling thread (the library call
 * site and, for CUDA errors, the CUDA error string); "" if none.  The string
 * is owned by the library and valid until the next failing call on the same
 * thread. */
const char *cc3_last_error(void);

/* ---------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Requests (residual or
 * Jacobian evaluations of problems of different size) are admitted while
 * others run, as slots and device memory free up; admitted requests keep
 * their inputs resident and their triple work interleaves on the GPU.
 * ------------------------------------------------------------------- */
typedef struct {
  int kind;               /* 0 = residual (Omega), 1 = Jacobian             */
  cc3_prec prec;
  int no, nv, naux;       /* sizes; naux may be 0 for kind 0                */
  const double *eps_o, *eps_v, *t2, *g_vvvo, *g_ooov, *g_ovov, *F_ov, *chol_L;
  int nvec;               /* kind 1: trial vectors                           */
  const double *omega, *R1, *R2;
  /* outputs (host pointers; filled by cc3_serve_wait) */
  double *Omega1, *Omega2, *E_T;  /* kind 0 */
  double *rho1, *rho2;            /* kind 1 */
  unsigned flags;                 /* context flags: 0 or CC3_DETERMINISTIC    */
} cc3_request;

typedef struct {
  long long submitted, admitted, completed, rejected, cancelled;
  double p50_ms, p99_ms, mean_ms;    /* submit -> completion latency        */
  double busy_s, wall_s;             /* device busy time, server wall time  */
  double nominal_flop;               /* over completed requests             */
  size_t hbm_in_use, hbm_peak;
} cc3_stats;

/* Starts a server on the current device with max_slots (1..64) worker
 * threads, each with its own CUDA stream; at most max_slots requests run at
 * once.  hbm_budget_bytes bounds the summed device footprint of the running
 * requests (0: 90 % of the free device memory at start). */
int cc3_serve_start(cc3_server **out, size_t hbm_budget_bytes, int max_slots);
/* Device bytes a request needs while it runs (inputs, workspace, the
 * Jacobian's intermediates and per-vector buffers); the admission test. */
int cc3_serve_footprint(const cc3_request *req, size_t *bytes);
/* Copies the request's inputs (host pointers) at submit and queues it;
 * returns a ticket.  CC3_ERR_BUSY if its footprint exceeds the budget (it
 * could never be admitted), CC3_ERR_ARG for an invalid request.  Admission is
 * first fit in arrival order, as slots and budget free up; a request that has
 * waited more than 10 s blocks later arrivals from overtaking it. */
int cc3_serve_submit(cc3_server *srv, const cc3_request *req, uint64_t *ticket);
/* *done = 1 once the request has completed, failed or been cancelled. */
int cc3_serve_poll(cc3_server *srv, uint64_t ticket, int *done);
/* Waits up to timeout_s (< 0: forever); writes the outputs into the pointers
 * given at submit, releases the ticket and returns the request's status
 * (CC3_ERR_TIMEOUT if it is still running: the ticket stays valid). */
int cc3_serve_wait(cc3_server *srv, uint64_t ticket, double timeout_s);
/* A queued request is dropped; a running one finishes on the device and its
 * result is discarded (wait then returns CC3_ERR_CANCELLED). */
int cc3_serve_cancel(cc3_server *srv, uint64_t ticket);
int cc3_serve_stats(cc3_server *srv, cc3_stats *out);
/* Cancels the queued requests, lets the running ones finish, joins the
 * workers and frees the server.  No other call on srv may be in progress or
 * follow. */
int cc3_serve_stop(cc3_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* CC3_H */
