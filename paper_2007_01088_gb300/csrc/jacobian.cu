// Right CC3 Jacobian transformation, triples part (paper: eq. "jcc3", the
// Jacobian paragraph of "Implementation", Algorithm 2), FP64 path.
//
// With H the T1-transformed Hamiltonian and R = (R1, R2) a trial vector at
// frequency w:
//   R3   = (w - eps)^{-1} P[ sum_d R^{ad}_{ij} g_{bdck} - sum_l R^{ab}_{il} g_{ljck}
//                           + sum_d t^{ad}_{ij} g^_{bdck} - sum_l t^{ab}_{il} g^_{ljck} ]
//   rho~ = contractions of R~3 with (g, F)      (as the residual, Algorithm 1)
//        + sum_c tau~ F^                        (the only tau~ term left in the loop)
//        + Z~v . R1 - Z~o . R1                   (Algorithm 2 intermediates, outside)
//   rho2 = (1/3) P^{ab}_{ij} (2 rho~ + rho~^{ba}),  rho1 = rho~1
// where g^ and F^ are the integrals differentiated along T1 = R1:
//   g^_{bdck} = -sum_l R^b_l (ld|ck) - sum_l R^c_l (bd|lk) + sum_e R^e_k (bd|ce)
//   g^_{ljck} =  sum_d R^d_j (ld|ck) - sum_m R^c_m (lj|mk) + sum_d R^d_k (lj|cd)
//   F^_{kc}   =  sum_ld [2 (kc|ld) - (kd|lc)] R^d_l
// (the vvvv integrals enter through the Cholesky vectors: sum_e R^e_k (bd|ce)
// = sum_J L^J_bd M^J_ck with M^J_ck = sum_e L^J_ce R^e_k).  tau~ is built once
// per triple and shared by all trial vectors of the call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cc3_internal.h"
#include "split.h"

namespace cc3 {
namespace {

#define CU(x)                                                              \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)
#define TRY(x)                   \
  do {                           \
    int r_ = (x);                \
    if (r_ != CC3_OK) return r_; \
  } while (0)

struct JacState {
  double *oooo = nullptr, *oovv = nullptr, *Zv = nullptr, *Zo = nullptr;
  double *wsWR = nullptr, *wsTTR = nullptr;
  int wsb = 0;
  bool blocks = false;
  int prep_prec = -1;  // precision the cached Z~v, Z~o were built in
};

JacState *jst(cc3_ctx *c) {
  if (!c->jac) c->jac = new (std::nothrow) JacState();
  return reinterpret_cast<JacState *>(c->jac);
}

int dalloc(double **p, size_t n) {
  *p = nullptr;
  if (cudaMalloc(p, sizeof(double) * (n ? n : 1)) != cudaSuccess) {
    cudaGetLastError();
    return CC3_FAIL(CC3_ERR_OOM, "Jacobian workspace");
  }
  return CC3_OK;
}

// Upload, launch and release one plan of one tile kind.
int run_plan(cc3_ctx *c, const Plan &p, int kind, const PtrTable &pt, cudaStream_t s) {
  if (p.jobs.empty()) return CC3_OK;
  DevPlan d;
  d.tile_kind = kind;
  TRY(upload_plan(p, &d, s));
  double f = 0.0;
  for (const Job &j : p.jobs)
    for (int t = 0; t < j.nterm; ++t)
      f += 2.0 * j.M * (double)j.N * p.terms[j.term0 + t].K * j.batch;
  trace_begin(c, TR_FP64_ENGINE, s);
  const int rc = launch_plan(d, pt, s, &c->counters.launches);
  trace_end(c, TR_FP64_ENGINE, s, f, 0.0);
  c->counters.executed_flop += f;
  cudaStreamSynchronize(s);  // the tables are freed next
  free_plan(&d);
  return rc;
}

static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};

int distinct_perms(const int ijk[3], int maps[6][3]) {
  int n = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return 0;
  for (int s = 0; s < 6; ++s) {
    bool dup = false;
    for (int u = 0; u < n; ++u)
      if (ijk[maps[u][0]] == ijk[PERM6[s][0]] && ijk[maps[u][1]] == ijk[PERM6[s][1]] &&
          ijk[maps[u][2]] == ijk[PERM6[s][2]])
        dup = true;
    if (!dup) {
      for (int k = 0; k < 3; ++k) maps[n][k] = PERM6[s][k];
      ++n;
    }
  }
  return n;
}

void fill_base(cc3_ctx *c, JacState *J, PtrTable *pt) {
  std::memset(pt, 0, sizeof(*pt));
  pt->p[B_T2] = c->t2;
  pt->p[B_VVVO] = c->vvvo;
  pt->p[B_OOVO] = c->oovo;
  pt->p[B_OOOV] = c->ooov;
  pt->p[B_OVOV] = c->ovov;
  pt->p[B_FOV] = c->F_ov;
  pt->p[B_EPSV] = c->eps_v;
  pt->p[B_EPSO] = c->eps_o;
  pt->p[B_WS_W] = c->ws_w;
  pt->p[B_WS_TT] = c->ws_tt;
  pt->p[B_WS_WR] = J->wsWR;
  pt->p[B_WS_TTR] = J->wsTTR;
  pt->p[B_ZV] = J->Zv;
  pt->p[B_ZO] = J->Zo;
  pt->p[B_OOOO] = J->oooo;
  pt->p[B_VVOO] = J->oovv;
  pt->p[B_CHOL] = c->chol;
  pt->p[B_SCRATCH] = c->omt;
}

// (lj|mk) and (lj|cd) from the Cholesky vectors, once per context
int ensure_blocks(cc3_ctx *c, JacState *J, cudaStream_t s) {
  if (J->blocks) return CC3_OK;
  const int no = c->no, nv = c->nv, n = no + nv;
  const long long n2 = (long long)n * n;
  TRY(dalloc(&J->oooo, (size_t)no * no * no * no));
  TRY(dalloc(&J->oovv, (size_t)no * no * nv * nv));
  PtrTable pt;
  fill_base(c, J, &pt);
  Plan P;
  const Opnd Loo = with_m2(op(B_CHOL, 0, 1, n2), no, n);  // rows (l, j), K = J
  int jb = new_job(P, 0, no * no, no * no, no * no, 1, 1, EPI_STORE);
  add_term(P, jb, Loo, Loo, c->naux);
  OutD o = out(B_OOOO, 0, (long long)no * no, 1);
  o.m_in = no;
  o.sm1 = (long long)no * no * no;
  o.n_in = no;
  o.sn1 = no;
  P.jobs[jb].C = o;
  P.jobs[jb].Ct = o;
  jb = new_job(P, 0, no * no, nv * nv, nv * nv, 1, 1, EPI_STORE);
  add_term(P, jb, Loo, with_m2(op(B_CHOL, (long long)no * n + no, 1, n2), nv, n), c->naux);
  o = out(B_VVOO, 0, (long long)nv * nv, 1);
  o.m_in = no;
  o.sm1 = (long long)no * nv * nv;
  o.n_in = nv;
  o.sn1 = nv;
  P.jobs[jb].C = o;
  P.jobs[jb].Ct = o;
  TRY(run_plan(c, P, 0, pt, s));
  J->blocks = true;
  return CC3_OK;
}

// tau and tau~ of one batch of triples (shared by the prep and the Jacobian)
int tau_batch(cc3_ctx *c, const PtrTable &pt, int t0, int t1, const std::vector<double> &eo,
              cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const TermSet set{B_T2, B_VVVO, B_OOVO};
  Plan pab, pc;
  for (int t = t0; t < t1; ++t) {
    const int *ijk = &c->tri_host[3 * t];
    const double e = eo[ijk[0]] + eo[ijk[1]] + eo[ijk[2]];
    plan_w_build(pab, no, nv, ijk, t - t0, B_WS_W, &set, 1, 0.0, e, 0);
    plan_w_build(pc, no, nv, ijk, t - t0, B_WS_W, &set, 1, 0.0, e, 1);
  }
  TRY(run_plan(c, pab, 0, pt, s));
  TRY(run_plan(c, pc, 0, pt, s));
  trace_begin(c, TR_FP64_ELEM, s);
  TRY(launch_contravariant(c->ws_w, c->ws_tt, nv, t1 - t0, s));
  trace_end(c, TR_FP64_ELEM, s, 0.0, 0.0);
  return CC3_OK;
}

// Algorithm 2: Zv[a][b][i][d] -= sum_c tau~^{abc}_{ijk} (jd|kc),
//              Zo[a][j][i][l] += sum_bc tau~^{abc}_{ijk} (lb|kc)
int ensure_prep(cc3_ctx *c, JacState *J, const std::vector<double> &eo, cudaStream_t s) {
  if (c->prep_valid && J->prep_prec == CC3_FP64) return CC3_OK;
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  if (!J->Zv) TRY(dalloc(&J->Zv, (size_t)nv3 * no));
  if (!J->Zo) TRY(dalloc(&J->Zo, (size_t)nv * no * no * no));
  TRY(launch_zero(J->Zv, (size_t)nv3 * no, s));
  TRY(launch_zero(J->Zo, (size_t)nv * no * no * no, s));
  PtrTable pt;
  fill_base(c, J, &pt);
  const long long st[3] = {nv2, nv, 1};
  for (int t0 = 0; t0 < c->ntri; t0 += c->batch) {
    const int t1 = std::min(c->ntri, t0 + c->batch);
    TRY(tau_batch(c, pt, t0, t1, eo, s));
    Plan pv, po;
    for (int t = t0; t < t1; ++t) {
      const int *ijk = &c->tri_host[3 * t];
      int maps[6][3];
      const int np = distinct_perms(ijk, maps);
      for (int u = 0; u < np; ++u) {
        const int *m = maps[u];
        const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
        const long long tt0 = (long long)(t - t0) * nv3;
        int jb = new_job(pv, 0, (int)nv2, nv, nv, 1, 1, EPI_ATOMIC);
        add_term(pv, jb, with_m2(op(B_WS_TT, tt0, st[m[1]], st[m[2]]), nv, st[m[0]]),
                 op(B_OVOV, (long long)q * nv * no * nv + (long long)r * nv, (long long)no * nv, 1, 0, 1),
                 nv);
        OutD o = out(B_ZV, (long long)p * nv, (long long)nv * no, 1);
        o.m_in = nv;
        o.sm1 = nv2 * no;
        pv.jobs[jb].C = o;
        pv.jobs[jb].Ct = o;
        jb = new_job(po, 1, nv, no, no, 1, 1, EPI_ATOMIC);
        add_term(po, jb, with_k2(op(B_WS_TT, tt0, st[m[0]], st[m[2]]), nv, st[m[1]]),
                 with_k2(op(B_OVOV, (long long)r * nv, (long long)nv * no * nv, 1), nv,
                         (long long)no * nv),
                 (int)nv2);
        o = out(B_ZO, ((long long)q * no + p) * no, (long long)no * no * no, 1);
        po.jobs[jb].C = o;
        po.jobs[jb].Ct = o;
      }
    }
    TRY(run_plan(c, pv, 0, pt, s));
    TRY(run_plan(c, po, 1, pt, s));
  }
  c->prep_valid = true;
  J->prep_prec = CC3_FP64;
  return CC3_OK;
}

// R1-dressed integrals of one trial vector (pointer table: B_R1, B_MJ,
// B_HVVVO, B_HOOVO, B_HF of that vector)
// chol = false leaves out the sum_J L^J_bd M^J_ck term of g^_vvvo (the split
// path adds it on the tensor cores) and starts g^_vvvo from zero instead.
int dress(cc3_ctx *c, const PtrTable &pt, cudaStream_t s, bool chol = true) {
  const int no = c->no, nv = c->nv, n = no + nv, naux = c->naux;
  const long long n2 = (long long)n * n, nv2 = (long long)nv * nv, nvo = (long long)nv * no;
  const long long ovovl = (long long)nv * no * nv;  // stride of l in ovov[l][d][k][c]
  Plan p0, pf, p1, p2, p3;
  // M^J_ck = sum_e L^J_ce R^e_k
  int jb = new_job(p0, 0, naux * nv, no, no, 1, 1, EPI_STORE);
  add_term(p0, jb, with_m2(op(B_CHOL, (long long)no * n + no, n, 1), nv, n2), op(B_R1, 0, nv, 1), nv);
  OutD o = out(B_MJ, 0, no, 1);
  o.m_in = nv;
  o.sm1 = nvo;
  p0.jobs[jb].C = o;
  p0.jobs[jb].Ct = o;
  // F^_kc = sum_ld [2 (kc|ld) - (kd|lc)] R^d_l   (one tail column, thin tiles)
  jb = new_job(pf, 1, no * nv, 1, 0, 1, 1, EPI_STORE);
  {
    const Opnd Bt = with_k2(op(B_R1, 0, 0, 1), nv, nv);
    const Opnd Aa = with_k2(with_m2(op(B_OVOV, 0, nvo, 1), nv, ovovl), nv, nv);
    const Opnd Ab = with_k2(with_m2(op(B_OVOV, 0, 1, nvo, 0, 1), nv, ovovl), nv, nv);
    add_term(pf, jb, Aa, Bt, no * nv, &Bt);
    add_term(pf, jb, Aa, Bt, no * nv, &Bt);
    add_term(pf, jb, Ab, Bt, no * nv, &Bt);
    o = out(B_HF, 0, 1, 0);
    o.m_in = nv;
    o.sm1 = nv;
    pf.jobs[jb].C = o;
    pf.jobs[jb].Ct = o;
  }
  TRY(run_plan(c, p0, 0, pt, s));
  TRY(run_plan(c, pf, 1, pt, s));
  // g^vvvo: Cholesky term (store), then the two R1 terms (accumulate)
  if (chol) {
    jb = new_job(p1, 0, (int)nv2, (int)nvo, (int)nvo, 1, 1, EPI_STORE);
    add_term(p1, jb, with_m2(op(B_CHOL, (long long)no * n + no, 1, n2), nv, n),
             with_m2(op(B_MJ, 0, 1, nvo), no, no), naux);
    o = out(B_HVVVO, 0, nvo, 1);
    o.m_in = nv;
    o.sm1 = nv2 * no;
    o.n_in = no;
    o.sn1 = no;
    p1.jobs[jb].C = o;
    p1.jobs[jb].Ct = o;
  } else {
    TRY(launch_zero(pt.p[B_HVVVO], (size_t)nv2 * nv * no, s));
  }
  // g^oovo: first term (store)
  jb = new_job(p1, 0, no, (int)nvo, (int)nvo, no, 1, EPI_STORE);
  add_term(p1, jb, op(B_R1, 0, nv, 1),
           with_m2(op(B_OVOV, 0, nv, nvo, ovovl), no, 1), nv);
  o = out(B_HOOVO, 0, nvo, 1, (long long)no * nv * no);
  o.n_in = no;
  o.sn1 = no;
  p1.jobs[jb].C = o;
  p1.jobs[jb].Ct = o;
  TRY(run_plan(c, p1, 0, pt, s));
  // - sum_l R^b_l (ld|ck)   (batch k)
  jb = new_job(p2, 0, nv, (int)nv2, (int)nv2, no, 1, EPI_ATOMIC);
  add_term(p2, jb, op(B_R1, 0, 1, nv, 0, 1), with_m2(op(B_OVOV, 0, 1, ovovl, nv), nv, nvo), no);
  o = out(B_HVVVO, 0, nv2 * no, no, 1);
  o.n_in = nv;
  o.sn1 = nvo;
  p2.jobs[jb].C = o;
  p2.jobs[jb].Ct = o;
  // - sum_l R^c_l (bd|lk) = - sum_l (lk|bd) R^c_l   (batch k)
  jb = new_job(p2, 0, (int)nv2, nv, nv, no, 1, EPI_ATOMIC);
  add_term(p2, jb, with_m2(op(B_VVOO, 0, 1, (long long)no * nv2, nv2), nv, nv),
           op(B_R1, 0, 1, nv, 0, 1), no);
  o = out(B_HVVVO, 0, nvo, no, 1);
  o.m_in = nv;
  o.sm1 = nv2 * no;
  p2.jobs[jb].C = o;
  p2.jobs[jb].Ct = o;
  // g^oovo: - sum_m R^c_m (lj|mk)   (batch k)
  jb = new_job(p2, 0, no * no, nv, nv, no, 1, EPI_ATOMIC);
  add_term(p2, jb, with_m2(op(B_OOOO, 0, (long long)no * no, no, 1), no, (long long)no * no * no),
           op(B_R1, 0, 1, nv, 0, 1), no);
  o = out(B_HOOVO, 0, nvo, no, 1);
  o.m_in = no;
  o.sm1 = (long long)no * nv * no;
  p2.jobs[jb].C = o;
  p2.jobs[jb].Ct = o;
  TRY(run_plan(c, p2, 0, pt, s));
  // g^oovo: + sum_d (lj|cd) R^d_k   (batch l)
  jb = new_job(p3, 1, (int)nvo, no, no, no, 1, EPI_ATOMIC);
  add_term(p3, jb, with_m2(op(B_VVOO, 0, nv, 1, (long long)no * nv2), nv, nv2), op(B_R1, 0, nv, 1),
           nv);
  o = out(B_HOOVO, 0, no, 1, (long long)no * nv * no);
  o.m_in = nv;
  o.sm1 = nvo;
  p3.jobs[jb].C = o;
  p3.jobs[jb].Ct = o;
  TRY(run_plan(c, p3, 1, pt, s));
  return CC3_OK;
}

}  // namespace

// FP64 Algorithm 2 intermediates (cached), tau and tau~ of a batch, and the
// base pointer table: shared with the left transformation (left.cu)
int jac_prep_fp64(cc3_ctx *c, cudaStream_t s) {
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  TRY(ensure_blocks(c, J, s));
  return ensure_prep(c, J, c->eo_h, s);
}
int jac_tau_batch(cc3_ctx *c, int t0, int t1, cudaStream_t s) {
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  PtrTable pt;
  fill_base(c, J, &pt);
  return tau_batch(c, pt, t0, t1, c->eo_h, s);
}
void jac_fill_ptrs(cc3_ctx *c, PtrTable *pt) {
  JacState *J = jst(c);
  if (J)
    fill_base(c, J, pt);
  else
    std::memset(pt, 0, sizeof(*pt));
}
// Upload, launch, free (FP64 engine), counted in the context's counters.
int jac_run_plan(cc3_ctx *c, const Plan &p, int kind, const PtrTable &pt, cudaStream_t s) {
  return run_plan(c, p, kind, pt, s);
}

int jac_blocks(cc3_ctx *c, cudaStream_t s) {
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  return ensure_blocks(c, J, s);
}

int jac_dress(cc3_ctx *c, const double *R1v, double *hv, double *ho, double *hf, double *mj,
              cudaStream_t s, bool chol) {
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  PtrTable pt;
  fill_base(c, J, &pt);
  pt.p[B_R1] = const_cast<double *>(R1v);
  pt.p[B_MJ] = mj;
  pt.p[B_HVVVO] = hv;
  pt.p[B_HOOVO] = ho;
  pt.p[B_HF] = hf;
  return dress(c, pt, s, chol);
}

int jac_z_buffers(cc3_ctx *c, double **Zv, double **Zo, bool zero, cudaStream_t s) {
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  const size_t nzv = (size_t)c->nv * c->nv * c->nv * c->no,
               nzo = (size_t)c->nv * c->no * c->no * c->no;
  if (!J->Zv) TRY(dalloc(&J->Zv, nzv));
  if (!J->Zo) TRY(dalloc(&J->Zo, nzo));
  if (zero) {
    TRY(launch_zero(J->Zv, nzv, s));
    TRY(launch_zero(J->Zo, nzo, s));
  }
  *Zv = J->Zv;
  *Zo = J->Zo;
  return CC3_OK;
}

void jac_set_prep(cc3_ctx *c, int prec) {
  JacState *J = jst(c);
  if (J) J->prep_prec = prec;
  c->prep_valid = prec >= 0;
}

int jac_prep_prec(cc3_ctx *c) {
  JacState *J = jst(c);
  return (J && c->prep_valid) ? J->prep_prec : -1;
}

// rho~[p][l][a][b] += sum_d Z~v[a][b][p][d] R1[l][d];
// rho~[p][q][a][d] -= sum_l Z~o[a][q][p][l] R1[l][d]
int jac_z_terms(cc3_ctx *c, const double *R1v, double *rtv, cudaStream_t s) {
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv;
  PtrTable pt;
  fill_base(c, J, &pt);
  pt.p[B_R1] = const_cast<double *>(R1v);
  pt.p[B_RHOT] = rtv;
  Plan pz1, pz0;
  for (int p = 0; p < no; ++p) {
    int jb = new_job(pz1, 1, (int)nv2, no, no, 1, 1, EPI_ATOMIC);
    add_term(pz1, jb, with_m2(op(B_ZV, (long long)p * nv, (long long)nv * no, 1), nv, nv2 * no),
             op(B_R1, 0, nv, 1), nv);
    OutD o = out(B_RHOT, (long long)p * no * nv2, 1, nv2);
    o.m_in = nv;
    o.sm1 = nv;
    pz1.jobs[jb].C = o;
    pz1.jobs[jb].Ct = o;
    jb = new_job(pz0, 0, nv * no, nv, nv, 1, 1, EPI_ATOMIC);
    add_term(pz0, jb,
             with_m2(op(B_ZO, (long long)p * no, (long long)no * no, 1, 0, 1), no,
                     (long long)no * no * no),
             op(B_R1, 0, 1, nv), no);
    o = out(B_RHOT, (long long)p * no * nv2, nv2, 1);
    o.m_in = no;
    o.sm1 = nv;
    pz0.jobs[jb].C = o;
    pz0.jobs[jb].Ct = o;
  }
  TRY(run_plan(c, pz1, 1, pt, s));
  TRY(run_plan(c, pz0, 0, pt, s));
  return CC3_OK;
}

int jacobian_fp64(cc3_ctx *c, int nvec, const double *w, const double *R1d, const double *R2d,
                  double *rho1d, double *rho2d, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv, nt2 = (long long)no * no * nv2;
  const long long nvvvo = nv3 * no, noovo = (long long)no * no * nv * no, n1 = (long long)no * nv;
  JacState *J = jst(c);
  if (!J) return CC3_ERR_OOM;
  TRY(ensure_blocks(c, J, s));
  std::vector<double> eo(no);
  CU(cudaMemcpyAsync(eo.data(), c->eps_o, sizeof(double) * no, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  // R3 slots: the bj triples of a batch for every vector (slot v * bj + t)
  const int bj = std::max(1, std::min(c->batch, c->batch / nvec));
  const int nslot = bj * nvec;
  if (J->wsb != nslot) {
    if (J->wsWR) cudaFree(J->wsWR);
    if (J->wsTTR) cudaFree(J->wsTTR);
    J->wsWR = J->wsTTR = nullptr;
    J->wsb = 0;
    TRY(dalloc(&J->wsWR, (size_t)nv3 * nslot));
    TRY(dalloc(&J->wsTTR, (size_t)nv3 * nslot));
    J->wsb = nslot;
  }
  TRY(ensure_prep(c, J, eo, s));
  // per-vector buffers
  double *hv = nullptr, *ho = nullptr, *hf = nullptr, *mj = nullptr, *rt = nullptr, *r1a = nullptr;
  int rc = CC3_OK;
  struct Guard {
    double **p[6];
    ~Guard() {
      for (double **q : p)
        if (*q) cudaFree(*q);
    }
  } guard{{&hv, &ho, &hf, &mj, &rt, &r1a}};
  TRY(dalloc(&hv, (size_t)nvvvo * nvec));
  TRY(dalloc(&ho, (size_t)noovo * nvec));
  TRY(dalloc(&hf, (size_t)n1 * nvec));
  TRY(dalloc(&mj, (size_t)c->naux * nv * no));
  TRY(dalloc(&rt, (size_t)nt2 * nvec));
  TRY(dalloc(&r1a, (size_t)n1 * nvec));
  TRY(launch_zero(rt, (size_t)nt2 * nvec, s));
  TRY(launch_zero(r1a, (size_t)n1 * nvec, s));
  PtrTable base;
  fill_base(c, J, &base);
  base.p[B_MJ] = mj;
  auto vec_ptrs = [&](int v) {
    PtrTable pt = base;
    pt.p[B_R1] = const_cast<double *>(R1d) + v * n1;
    pt.p[B_R2] = const_cast<double *>(R2d) + v * nt2;
    pt.p[B_HVVVO] = hv + v * nvvvo;
    pt.p[B_HOOVO] = ho + v * noovo;
    pt.p[B_HF] = hf + v * n1;
    pt.p[B_RHOT] = rt + v * nt2;
    pt.p[B_RHO1] = r1a + v * n1;
    return pt;
  };
  for (int v = 0; v < nvec; ++v) TRY(dress(c, vec_ptrs(v), s));
  // one launch per phase for all vectors: the vector's part of each per-vector
  // buffer is an offset added to the jobs planned for it (buffers of vector 0
  // in the pointer table)
  const PtrTable all = vec_ptrs(0);
  auto shift = [&](Plan &P, size_t j0, size_t k0, int v) {
    long long off[B_COUNT] = {0};
    off[B_R2] = v * nt2;
    off[B_HVVVO] = v * nvvvo;
    off[B_HOOVO] = v * noovo;
    off[B_HF] = v * n1;
    off[B_RHOT] = v * nt2;
    off[B_RHO1] = v * n1;
    for (size_t j = j0; j < P.jobs.size(); ++j) {
      P.jobs[j].C.off += off[P.jobs[j].C.buf];
      P.jobs[j].Ct.off += off[P.jobs[j].Ct.buf];
    }
    for (size_t k = k0; k < P.terms.size(); ++k) {
      P.terms[k].A.off += off[P.terms[k].A.buf];
      P.terms[k].B.off += off[P.terms[k].B.buf];
      P.terms[k].Bt.off += off[P.terms[k].Bt.buf];
    }
  };
  const TermSet sets[2] = {{B_R2, B_VVVO, B_OOVO}, {B_T2, B_HVVVO, B_HOOVO}};
  for (int t0 = 0; t0 < c->ntri; t0 += bj) {
    const int t1 = std::min(c->ntri, t0 + bj);
    TRY(tau_batch(c, base, t0, t1, eo, s));
    Plan pF, pab, pc, pom, pth;
    for (int v = 0; v < nvec; ++v)
      for (int t = t0; t < t1; ++t) {
        const int *ijk = &c->tri_host[3 * t];
        const int u = v * bj + (t - t0);
        const double e = eo[ijk[0]] + eo[ijk[1]] + eo[ijk[2]];
        size_t j0 = pF.jobs.size(), k0 = pF.terms.size();
        plan_omega_contractions(pF, no, nv, ijk, t - t0, B_WS_TT, B_OVOV, B_HF, B_OOOV, true,
                                B_VVVO, B_RHOT, B_RHO1, 1, 4);
        shift(pF, j0, k0, v);
        j0 = pab.jobs.size(), k0 = pab.terms.size();
        plan_w_build(pab, no, nv, ijk, u, B_WS_WR, sets, 2, 0.0, 0.0, 0);
        shift(pab, j0, k0, v);
        j0 = pc.jobs.size(), k0 = pc.terms.size();
        plan_w_build(pc, no, nv, ijk, u, B_WS_WR, sets, 2, w[v], e, 1);
        shift(pc, j0, k0, v);
        j0 = pom.jobs.size(), k0 = pom.terms.size();
        plan_omega_contractions(pom, no, nv, ijk, u, B_WS_TTR, B_OVOV, B_FOV, B_OOOV, true,
                                B_VVVO, B_RHOT, B_RHO1, 2, 1);
        shift(pom, j0, k0, v);
        j0 = pth.jobs.size(), k0 = pth.terms.size();
        plan_omega_contractions(pth, no, nv, ijk, u, B_WS_TTR, B_OVOV, B_FOV, B_OOOV, true,
                                B_VVVO, B_RHOT, B_RHO1, 1, 2);
        shift(pth, j0, k0, v);
      }
    TRY(run_plan(c, pF, 1, all, s));
    TRY(run_plan(c, pab, 0, all, s));
    TRY(run_plan(c, pc, 0, all, s));
    trace_begin(c, TR_FP64_ELEM, s);
    TRY(launch_contravariant(J->wsWR, J->wsTTR, nv, nslot, s));
    trace_end(c, TR_FP64_ELEM, s, 0.0, 0.0);
    TRY(run_plan(c, pom, 0, all, s));
    TRY(run_plan(c, pth, 1, all, s));
  }
  // Z~v . R1 and Z~o . R1 (outside the triple loop), back-transform
  for (int v = 0; v < nvec; ++v) {
    TRY(jac_z_terms(c, R1d + v * n1, rt + v * nt2, s));
    TRY(launch_back_transform(rt + v * nt2, rho2d + v * nt2, no, nv, s));
    CU(cudaMemcpyAsync(rho1d + v * n1, r1a + v * n1, sizeof(double) * n1,
                       cudaMemcpyDeviceToDevice, s));
  }
  CU(cudaStreamSynchronize(s));
  return rc;
}

// Device bytes of the Jacobian's cached blocks, Algorithm 2 intermediates,
// R3 workspace and per-call buffers (the same arithmetic as the allocations
// above), for admission control.
size_t jacobian_footprint(int no, int nv, int naux, int nvec, int ntri, bool host_io) {
  const size_t nv3 = (size_t)nv * nv * nv, nt2 = (size_t)no * no * nv * nv,
               n1 = (size_t)no * nv, o4 = (size_t)no * no * no * no;
  size_t d = o4 + nt2;                               // oooo, oovv
  d += nv3 * no + (size_t)nv * no * no * no;         // Zv, Zo
  d += 2 * nv3 * std::max(nvec, batch_for(nv, ntri));  // R3 workspace (all vectors' slots)
  d += (size_t)nvec * (nv3 * no + (size_t)no * no * nv * no + n1 + nt2 + n1);  // per vector
  d += (size_t)naux * nv * no;                       // M^J_ck
  if (host_io) d += (size_t)nvec * 2 * (n1 + nt2);   // staging of R and rho
  const size_t plans = (size_t)std::max(1, ntri) * 24 * (sizeof(Job) + 2 * sizeof(Term));
  return d * sizeof(double) + plans + 4096;
}

void jacobian_destroy(cc3_ctx *c) {
  JacState *J = reinterpret_cast<JacState *>(c->jac);
  if (!J) return;
  double *b[] = {J->oooo, J->oovv, J->Zv, J->Zo, J->wsWR, J->wsTTR};
  for (double *p : b)
    if (p) cudaFree(p);
  delete J;
  c->jac = nullptr;
}

}  // namespace cc3

extern "C" int cc3_jacobian_triples(cc3_ctx *c, cc3_prec prec, int nvec, const double *omega,
                                    const double *R1, const double *R2, double *rho1,
                                    double *rho2, void *cuda_stream) {
  using namespace cc3;
  if (!c || nvec < 1 || !omega || !R1 || !R2 || !rho1 || !rho2) return CC3_ERR_ARG;
  if (c->general)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "the Jacobian needs symmetric integrals");
  if (c->naux < 1 || !c->chol)
    return CC3_FAIL(CC3_ERR_ARG, "the Jacobian needs the Cholesky vectors (chol_L)");
  if (prec == CC3_SPLIT_INT8) return CC3_ERR_UNSUPPORTED;
  if (c->flags & CC3_DETERMINISTIC)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "deterministic reductions cover the residual only");
  if (prec != CC3_FP64 && prec != CC3_SPLIT_BF16) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  // the R3 denominators (w - eps^{abc}_{ijk}) of every vector stay away from 0
  // (host check on the context's copies of the orbital energies, before any
  // device work)
  for (int v = 0; v < nvec; ++v) {
    if (!std::isfinite(omega[v])) return CC3_FAIL(CC3_ERR_ARG, "non-finite frequency");
    bool seen = false;
    for (int u = 0; u < v; ++u) seen = seen || omega[u] == omega[v];
    if (seen || c->ntri == 0) continue;
    const double gap = denominator_gap(c->no, c->nv, c->eo_h.data(), c->ev_h.data(), c->ntri,
                                       c->tri_host.data(), omega[v]);
    if (gap < CC3_DENOM_MIN)
      return CC3_FAIL(CC3_ERR_DENOM, "a frequency lies within CC3_DENOM_MIN of a triples "
                                     "denominator");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int no = c->no, nv = c->nv;
  const size_t n1 = (size_t)no * nv, nt2 = (size_t)no * no * nv * nv;
  long long wsum = 0;
  for (int t = 0; t < c->ntri; ++t) {
    const int *x = &c->tri_host[3 * t];
    wsum += (x[0] == x[1] && x[1] == x[2]) ? 0 : ((x[0] != x[1] && x[1] != x[2]) ? 6 : 3);
  }
  c->counters = cc3_counters{};
  trace_reset(c);
  c->counters.nominal_flop = 8.0 * (double)nv * nv * nv * nv * (double)wsum * nvec;
  const bool dev = (c->flags & CC3_DEVICE_PTRS) != 0;
  double *dR1 = const_cast<double *>(R1), *dR2 = const_cast<double *>(R2), *dr1 = rho1,
         *dr2 = rho2;
  std::vector<double *> tmp;
  auto mk = [&](double **p, size_t n) {
    if (cudaMalloc(p, sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    tmp.push_back(*p);
    return true;
  };
  int rc = CC3_OK;
  if (!dev) {
    if (!mk(&dR1, n1 * nvec) || !mk(&dR2, nt2 * nvec) || !mk(&dr1, n1 * nvec) ||
        !mk(&dr2, nt2 * nvec))
      rc = CC3_FAIL(CC3_ERR_OOM, "Jacobian staging");
    if (rc == CC3_OK &&
        (cudaMemcpyAsync(dR1, R1, sizeof(double) * n1 * nvec, cudaMemcpyHostToDevice, s) !=
             cudaSuccess ||
         cudaMemcpyAsync(dR2, R2, sizeof(double) * nt2 * nvec, cudaMemcpyHostToDevice, s) !=
             cudaSuccess))
      rc = CC3_FAIL(CC3_ERR_CUDA, "Jacobian upload");
  }
  if (rc == CC3_OK) {
    if (prec == CC3_FP64)
      rc = jacobian_fp64(c, nvec, omega, dR1, dR2, dr1, dr2, s);
    else
      rc = split_jacobian(c, nvec, omega, dR1, dR2, dr1, dr2, s);
  }
  if (rc == CC3_OK && !dev) {
    if (cudaMemcpyAsync(rho1, dr1, sizeof(double) * n1 * nvec, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(rho2, dr2, sizeof(double) * nt2 * nvec, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = CC3_FAIL(CC3_ERR_CUDA, "Jacobian download");
  }
  cudaStreamSynchronize(s);
  for (double *p : tmp) cudaFree(p);
  if (rc == CC3_OK) rc = trace_collect(c, s);
  return rc;
}
