// Internal declarations of libcc3 (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/cc3.h"

namespace cc3 {

// ---------------------------------------------------------------------------
// Strided operand of a contraction: element (m, k) of an M x K matrix sits at
//   base[buf] + off + batch*sb + (m / m_in)*sm1 + (m % m_in)*sm0
//                              + (k / k_in)*sk1 + (k % k_in)*sk0
// (two-level row and column indices cover the permuted views of the nv^3
// triples amplitudes and the integral blocks without reordering them).
// ---------------------------------------------------------------------------
struct Opnd {
  int buf;
  int m_in, k_in;
  int neg;  // 1: operand enters with a minus sign
  long long off, sb, sm1, sm0, sk1, sk0;
};

// One term of a multi-term contraction C[m][n] += sum_k A[m][k] * B[n][k].
// Columns n >= Job::Nm take their B values from Bt (the "tail" columns, e.g.
// the singles contraction riding along with the vvov contraction).
struct Term {
  Opnd A, B, Bt;
  int K;
};

struct OutD {
  int buf;
  int m_in, n_in;
  long long off, sb, sm1, sm0, sn1, sn0;
};

enum EpiMode { EPI_STORE = 0, EPI_ATOMIC = 1, EPI_TAU = 2 };

struct Job {
  int M, N, Nm, batch;
  int term0, nterm;
  int tiles_m, tiles_n, ksplit;
  int mode;
  long long tile_base;  // first CTA of this job within its launch
  OutD C, Ct;           // main and tail outputs
  // EPI_TAU: C = (C + acc) / (w - eps), eps = ev[m] + ev[n / nv] + ev[n % nv] - eo
  double w, eo;
};

enum { MAX_BUFS = 32 };
struct PtrTable {
  double *p[MAX_BUFS];
  // deterministic mode: accumulating outputs go to 128-bit fixed point
  // (lo, hi word pairs per element) instead of FP64 atomics when set
  unsigned long long *fx[MAX_BUFS];
};

// Buffer ids of the pointer table.
enum BufId {
  B_T2 = 0, B_VVVO, B_OOVO, B_OOOV, B_OVOV, B_FOV, B_EPSV, B_EPSO,
  B_WS_W, B_WS_TT, B_OMT, B_OM1,
  B_R2, B_HVVVO, B_HOOVO, B_HF, B_ZV, B_ZO, B_VVOO, B_OOOO,
  B_RHOT, B_RHO1, B_TT_TAU, B_SCRATCH, B_SLOTEXP,
  B_WS_WR, B_WS_TTR, B_MJ, B_CHOL, B_R1, B_WS_W3, B_VVOV,
  B_COUNT,
  // the left transformation (left.cu) reuses slots the right one does not
  // touch there: Lt2, sigma1, sigma2 (before symmetrising), G, H, Q
  B_LT = B_R2, B_S1 = B_RHO1, B_S2 = B_RHOT, B_G = B_HVVVO, B_H = B_HOOVO, B_Q = B_HF,
  // the densities (density.cu) reuse Lt2 and Q (= Dov) as above, and take
  // Y, Dvv and the virtual loop's two bracket buffers from unused slots
  B_DY = B_ZV, B_DVV = B_ZO, B_DOV = B_Q, B_VBT = B_VVOO, B_VBX = B_OOOO
};
static_assert((int)B_COUNT <= (int)MAX_BUFS, "pointer table");

struct Plan {  // a host-built list of jobs for one launch
  std::vector<Job> jobs;
  std::vector<Term> terms;
  long long tiles = 0;
};

struct DevPlan {  // the same, resident on the device
  Job *jobs = nullptr;
  Term *terms = nullptr;
  int njobs = 0;
  long long tiles = 0;
  int tile_kind = 0;  // 0: 64x64 tiles, 1: 128x4 thin tiles
  double flop = 0.0;  // useful FLOP of the launch
};

// Kernel classes of the tracer.
enum TraceClass {
  TR_FP64_ENGINE = 0, TR_FP64_ELEM, TR_SPLIT_W, TR_SPLIT_OMEGA, TR_SPLIT_ELEM, TR_OUTPUT,
  TR_NCLASS
};
struct Tracer {
  bool on = false;
  std::vector<cudaEvent_t> ev[TR_NCLASS];  // start/stop pairs
  int used[TR_NCLASS] = {0};
  long long launches[TR_NCLASS] = {0};
  double flop[TR_NCLASS] = {0}, slice_flop[TR_NCLASS] = {0}, ms[TR_NCLASS] = {0};
};

}  // namespace cc3

struct cc3_ctx {
  int no = 0, nv = 0, naux = 0;
  unsigned flags = 0;
  int device = 0;
  cudaStream_t stream0 = nullptr;
  // device copies (FP64)
  double *eps_o = nullptr, *eps_v = nullptr, *t2 = nullptr, *vvvo = nullptr,
         *oovo = nullptr, *ooov = nullptr, *ovov = nullptr, *F_ov = nullptr,
         *chol = nullptr, *vvoo = nullptr, *oooo = nullptr;
  // general (T1-transformed) integrals: vvov[d][b][k][c] = g_dbkc and oovo
  // given on their own instead of derived from vvvo and ooov by the 8-fold
  // symmetry (cc3_ctx_create_general); vvov is null for symmetric contexts
  double *vvov = nullptr;
  bool general = false;
  // host copies of the orbital energies (denominator checks, plan epilogues)
  std::vector<double> eo_h, ev_h;
  // triple list (device and host), weights
  std::vector<int> tri_host;  // 3 per triple
  int ntri = 0;
  // workspace
  int batch = 0;  // triples per batch
  double *ws_w = nullptr, *ws_tt = nullptr, *ws_tt2 = nullptr;
  double *omt = nullptr, *om1 = nullptr;
  unsigned long long *omt_fx = nullptr, *om1_fx = nullptr;  // deterministic mode
  // Jacobian cache (Algorithm 2 intermediates)
  double *Zv = nullptr, *Zo = nullptr;
  bool prep_valid = false;
  // Jacobian scratch (per call)
  double *R2 = nullptr, *hvvvo = nullptr, *hoovo = nullptr, *hF = nullptr,
         *rhot = nullptr, *rho1 = nullptr, *Mj = nullptr;
  void *jac = nullptr;  // Jacobian state private to jacobian.cu
  // driver state private to api.cu / split path state private to split.cu
  void *ext = nullptr;
  void *split = nullptr;
  int slices = 0;
  // counters and tracing
  cc3_counters counters{};
  cc3::Tracer trace;
  // device status word (bounded waits)
  int *status = nullptr;
  std::mutex mu;
};

namespace cc3 {
// tracing helpers (api.cu): bracket one launch of class `cls`
void trace_begin(cc3_ctx *c, int cls, cudaStream_t s);
void trace_end(cc3_ctx *c, int cls, cudaStream_t s, double flop, double slice_flop);
void trace_reset(cc3_ctx *c);
int trace_collect(cc3_ctx *c, cudaStream_t s);
// failure detail for cc3_last_error (api.cu); returns `status`
int record_error(int status, const char *file, int line, const char *what);
#define CC3_FAIL(status, what) ::cc3::record_error((status), __FILE__, __LINE__, (what))

// engine (fp64_engine.cu)
int upload_plan(const Plan &p, DevPlan *d, cudaStream_t s);
void free_plan(DevPlan *d);
int launch_plan(const DevPlan &d, const PtrTable &ptrs, cudaStream_t s,
                long long *launches);

// misc kernels (kernels.cu)
int launch_contravariant(const double *tau_cab, double *tt_abc, int nv,
                         int nslot, cudaStream_t s);
int launch_back_transform(const double *omt, double *om2, int no, int nv,
                          cudaStream_t s);
int launch_energy(const double *t2, const double *omt, double *E, int no,
                  int nv, cudaStream_t s);
int launch_transpose_ooov_to_oovo(const double *ooov, double *oovo, int no,
                                  int nv, cudaStream_t s);
int launch_zero(double *p, size_t n, cudaStream_t s);
// out[i] = the 128-bit fixed-point value fx[2i..2i+1] as a double
int launch_fx_to_double(const unsigned long long *fx, double *out, size_t n, cudaStream_t s);

// plans (plans.cu): operand / output descriptors and job builders
Opnd op(int buf, long long off, long long sm0, long long sk0, long long sb = 0, int neg = 0);
Opnd with_m2(Opnd o, int m_in, long long sm1);
Opnd with_k2(Opnd o, int k_in, long long sk1);
OutD out(int buf, long long off, long long sm0, long long sn0, long long sb = 0);
// kind 0: 64 x 64 tiles, kind 1: 256 x 4 tiles
int new_job(Plan &P, int kind, int M, int N, int Nm, int batch, int ksplit, int mode);
void add_term(Plan &P, int job, const Opnd &A, const Opnd &B, int K, const Opnd *Bt = nullptr);
struct TermSet { int bt, bv, bo; };  // (t-like, vvvo-like, oovo-like) buffers
void plan_w_build(Plan &P, int no, int nv, const int ijk[3], int slot,
                  int buf_w, const TermSet *sets, int nsets, double w,
                  double eo, int phase);
void plan_omega_contractions(Plan &P, int no, int nv, const int ijk[3],
                             int slot, int buf_tt, int buf_ovov, int buf_fov,
                             int buf_ooov, bool vvov_from_vvvo, int buf_vvov,
                             int buf_omt, int buf_om1, int ksplit, int which);
double nominal_flop_omega(int no, int nv, int ntri_weighted);

// Jacobian state (jacobian.cu)
void jacobian_destroy(cc3_ctx *c);
// pieces shared by the FP64 and split Jacobians (jacobian.cu)
int jac_blocks(cc3_ctx *c, cudaStream_t s);  // (lj|mk), (lj|cd) from the Cholesky vectors
// g^_vvvo, g^_oovo, F^ and M^J_ck of one trial vector (FP64); chol = false
// leaves the Cholesky (vvvv) term of g^_vvvo to the caller
int jac_dress(cc3_ctx *c, const double *R1v, double *hv, double *ho, double *hf, double *mj,
              cudaStream_t s, bool chol = true);
int jac_z_buffers(cc3_ctx *c, double **Zv, double **Zo, bool zero, cudaStream_t s);
void jac_set_prep(cc3_ctx *c, int prec);  // the cached Z~ are valid, built in prec
int jac_prep_prec(cc3_ctx *c);            // -1 if the cache is not valid
int jac_z_terms(cc3_ctx *c, const double *R1v, double *rtv, cudaStream_t s);
int jac_prep_fp64(cc3_ctx *c, cudaStream_t s);           // cached FP64 Z~v, Z~o
int jac_tau_batch(cc3_ctx *c, int t0, int t1, cudaStream_t s);  // tau~ -> ws_tt
void jac_fill_ptrs(cc3_ctx *c, PtrTable *pt);
int jac_run_plan(cc3_ctx *c, const Plan &p, int kind, const PtrTable &pt, cudaStream_t s);
// pieces of the left transformation shared with the densities (left.cu):
// Q[r][z] += sum_xy Lt2[p][q][x][y] tau~[x][y][z] jobs of one triple, and the
// covariant L3 (wsW, [c][a][b] per slot) with its contravariant form (wsT)
void plan_left_q(Plan &P, int no, int nv, const int ijk[3], int slot);
int left_l3_batch(cc3_ctx *c, const PtrTable &pt, int t0, int t1, double w, const double *L1d,
                  const double *ltd, int *tri, double *wsW, double *wsT, cudaStream_t s);
int left_finish(cc3_ctx *c, const PtrTable &pt, const double *s2raw, double *s2d,
                cudaStream_t s, bool chol_done = false);
// the densities' FP64 pieces shared by both paths (density.cu): the end of the
// occupied loop (pt: B_DY = Y, B_DOV = Dov, B_T2), and Doo from tau and L~ of
// every triple of tri (3 ints each, sorted i >= j >= k) held resident
int density_tail(cc3_ctx *c, const PtrTable &pt, double *Dvv, cudaStream_t s);
int density_doo_resident(cc3_ctx *c, const float2 *tau_all, const float2 *lt_all,
                         const std::vector<int> &tri, double *Doo, cudaStream_t s);

// smallest |w - eps^{abc}_{ijk}| over every (a, b, c) and the ntri triples
// ijk (host arrays; ntri = 0: the full loop); api.cu
double denominator_gap(int no, int nv, const double *eo, const double *ev, int ntri,
                       const int *ijk, double w);

// device footprints for admission control (api.cu, jacobian.cu)
int batch_for(int nv, int ntri);
size_t ctx_footprint(int no, int nv, int naux, int ntri, bool host_io);
size_t jacobian_footprint(int no, int nv, int naux, int nvec, int ntri, bool host_io);
}  // namespace cc3
