// C ABI of libcc3: context, staging, the triple loop driver of the residual
// (paper, Algorithm 1) and error strings.  Device work only: no CPU
// fallback exists in this library.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cc3_internal.h"
#include "split.h"

using namespace cc3;

#define CU(x)                                                          \
  do {                                                                 \
    cudaError_t e_ = (x);                                              \
    if (e_ != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)
#define TRY(x)              \
  do {                      \
    int r_ = (x);           \
    if (r_ != CC3_OK) return r_; \
  } while (0)

namespace {

struct OmegaPlans {
  std::vector<DevPlan> ab, c, om, thin;
  std::vector<int> nslot;  // triples per batch
  double executed = 0.0;
  bool valid = false;
};

struct CtxExtra {
  OmegaPlans omega;
  double *escr = nullptr;   // 257 doubles: energy + partials
  double *om2tmp = nullptr; // host-pointer mode output staging
};

CtxExtra *extra(cc3_ctx *c) { return reinterpret_cast<CtxExtra *>(c->ext); }

cudaMemcpyKind in_kind(const cc3_ctx *c) {
  return (c->flags & CC3_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                      : cudaMemcpyHostToDevice;
}
cudaMemcpyKind out_kind(const cc3_ctx *c) {
  return (c->flags & CC3_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                      : cudaMemcpyDeviceToHost;
}

int dalloc(double **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc(p, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return CC3_ERR_OOM;
  }
  return CC3_OK;
}

void free_omega_plans(OmegaPlans &P) {
  for (auto *v : {&P.ab, &P.c, &P.om, &P.thin})
    for (auto &d : *v) free_plan(&d);
  P.ab.clear(); P.c.clear(); P.om.clear(); P.thin.clear(); P.nslot.clear();
  P.valid = false;
}

double plan_flops(const Plan &P) {
  double f = 0.0;
  for (const Job &j : P.jobs)
    for (int t = 0; t < j.nterm; ++t)
      f += 2.0 * j.M * (double)j.N * P.terms[j.term0 + t].K * j.batch;
  return f;
}

int weight_of(const int *ijk) {
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return 0;
  if (ijk[0] != ijk[1] && ijk[1] != ijk[2] && ijk[0] != ijk[2]) return 6;
  return 3;
}

void fill_ptrs(cc3_ctx *c, PtrTable *pt) {
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
  pt->p[B_OMT] = c->omt;
  pt->p[B_OM1] = c->om1;
  pt->p[B_SCRATCH] = c->omt;
  pt->p[B_VVOV] = c->vvov;
  pt->fx[B_OMT] = c->omt_fx;  // null unless CC3_DETERMINISTIC
  pt->fx[B_OM1] = c->om1_fx;
}

int build_omega_plans(cc3_ctx *c, cudaStream_t s) {
  CtxExtra *X = extra(c);
  OmegaPlans &OP = X->omega;
  free_omega_plans(OP);
  const int no = c->no, nv = c->nv;
  std::vector<double> eo(c->no);
  CU(cudaMemcpy(eo.data(), c->eps_o, sizeof(double) * no, cudaMemcpyDeviceToHost));
  const TermSet set{B_T2, B_VVVO, B_OOVO};
  double executed = 0.0;
  for (int t0 = 0; t0 < c->ntri; t0 += c->batch) {
    const int t1 = std::min(c->ntri, t0 + c->batch);
    Plan pab, pc, pom, pth;
    for (int t = t0; t < t1; ++t) {
      const int *ijk = &c->tri_host[3 * t];
      const int slot = t - t0;
      const double e = eo[ijk[0]] + eo[ijk[1]] + eo[ijk[2]];
      plan_w_build(pab, no, nv, ijk, slot, B_WS_W, &set, 1, 0.0, e, 0);
      plan_w_build(pc, no, nv, ijk, slot, B_WS_W, &set, 1, 0.0, e, 1);
      // vvov: its own block for general integrals, else a view of vvvo
      plan_omega_contractions(pom, no, nv, ijk, slot, B_WS_TT, B_OVOV, B_FOV,
                              B_OOOV, !c->general, c->general ? B_VVOV : B_VVVO, B_OMT,
                              B_OM1, 2, 1);
      plan_omega_contractions(pth, no, nv, ijk, slot, B_WS_TT, B_OVOV, B_FOV,
                              B_OOOV, !c->general, c->general ? B_VVOV : B_VVVO, B_OMT,
                              B_OM1, 1, 2);
    }
    executed += plan_flops(pab) + plan_flops(pc) + plan_flops(pom) + plan_flops(pth);
    DevPlan d;
    d.tile_kind = 0;
    OP.ab.push_back(d); OP.c.push_back(d); OP.om.push_back(d);
    d.tile_kind = 1;
    OP.thin.push_back(d);
    TRY(upload_plan(pab, &OP.ab.back(), s));
    TRY(upload_plan(pc, &OP.c.back(), s));
    TRY(upload_plan(pom, &OP.om.back(), s));
    TRY(upload_plan(pth, &OP.thin.back(), s));
    OP.ab.back().flop = plan_flops(pab);
    OP.c.back().flop = plan_flops(pc);
    OP.om.back().flop = plan_flops(pom);
    OP.thin.back().flop = plan_flops(pth);
    OP.ab.back().tile_kind = 0; OP.c.back().tile_kind = 0;
    OP.om.back().tile_kind = 0; OP.thin.back().tile_kind = 1;
    OP.nslot.push_back(t1 - t0);
  }
  OP.executed = executed;
  OP.valid = true;
  return CC3_OK;
}

int default_triples(cc3_ctx *c) {
  c->tri_host.clear();
  for (int i = 0; i < c->no; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k) {
        if (i == j && j == k) continue;
        c->tri_host.push_back(i);
        c->tri_host.push_back(j);
        c->tri_host.push_back(k);
      }
  c->ntri = (int)(c->tri_host.size() / 3);
  return CC3_OK;
}

int choose_batch(cc3_ctx *c) { return batch_for(c->nv, c->ntri); }

int alloc_workspace(cc3_ctx *c) {
  const size_t nv3 = (size_t)c->nv * c->nv * c->nv;
  if (c->ws_w) cudaFree(c->ws_w);
  if (c->ws_tt) cudaFree(c->ws_tt);
  c->ws_w = c->ws_tt = nullptr;
  TRY(dalloc(&c->ws_w, nv3 * c->batch));
  TRY(dalloc(&c->ws_tt, nv3 * c->batch));
  return CC3_OK;
}

}  // namespace

namespace cc3 {
// Triples per batch of the FP64 path: two nv^3 buffers per triple in flight,
// about 4 GB in all, at most 32.
int batch_for(int nv, int ntri) {
  const double nv3b = (double)nv * nv * nv * sizeof(double);
  int b = (int)std::max(1.0, std::min(32.0, 4.0e9 / (2.0 * nv3b)));
  return std::min(b, std::max(1, ntri));
}

// Device bytes held by a context after cc3_ctx_create and one FP64 residual
// call (inputs, the oovo copy, outputs, the FP64 workspace and plan tables).
size_t ctx_footprint(int no, int nv, int naux, int ntri, bool host_io) {
  const size_t nt2 = (size_t)no * no * nv * nv, nvvvo = (size_t)nv * nv * nv * no,
               nooov = (size_t)no * no * no * nv, n = (size_t)no + nv;
  size_t d = no + nv + nt2 + nvvvo + 2 * nooov + nt2 + (size_t)no * nv;  // inputs + oovo
  d += (size_t)naux * n * n;
  d += nt2 + (size_t)no * nv + 257;  // omt, om1, energy scratch
  if (host_io) d += nt2;             // Omega2 staging
  d += 2 * (size_t)nv * nv * nv * batch_for(nv, ntri);
  const size_t plans = (size_t)std::max(1, ntri) * 8 * (sizeof(Job) + 2 * sizeof(Term));
  return d * sizeof(double) + plans + 4096;
}

// Smallest |w - eps^{abc}_{ijk}| with eps^{abc}_{ijk} = e_a + e_b + e_c - e_i
// - e_j - e_k, over every virtual triple (a, b, c) (all nv^3 of them enter
// the division) and the occupied triples of the loop.  The sorted pair sums
// e_b + e_c (b <= c) turn the search over (a, b, c) into nv binary searches
// per occupied triple.
double denominator_gap(int no, int nv, const double *eo, const double *ev, int ntri,
                       const int *ijk, double w) {
  std::vector<double> pair;
  pair.reserve((size_t)nv * (nv + 1) / 2);
  for (int b = 0; b < nv; ++b)
    for (int c = b; c < nv; ++c) pair.push_back(ev[b] + ev[c]);
  std::sort(pair.begin(), pair.end());
  double gap = 1e300;
  auto one = [&](int i, int j, int k) {
    const double T = w + eo[i] + eo[j] + eo[k];  // e_a + e_b + e_c closest to T
    for (int a = 0; a < nv; ++a) {
      const double x = T - ev[a];
      const auto it = std::lower_bound(pair.begin(), pair.end(), x);
      if (it != pair.end()) gap = std::min(gap, std::fabs(*it - x));
      if (it != pair.begin()) gap = std::min(gap, std::fabs(*(it - 1) - x));
    }
  };
  if (ntri > 0 && ijk) {
    for (int t = 0; t < ntri; ++t) one(ijk[3 * t], ijk[3 * t + 1], ijk[3 * t + 2]);
  } else {
    for (int i = 0; i < no; ++i)
      for (int j = 0; j <= i; ++j)
        for (int k = 0; k <= j; ++k)
          if (!(i == j && j == k)) one(i, j, k);
  }
  return gap;
}

static thread_local char g_last_error[512] = "";
int record_error(int status, const char *file, int line, const char *what) {
  const char *base = std::strrchr(file, '/');
  std::snprintf(g_last_error, sizeof(g_last_error), "%s:%d: %s (%s)", base ? base + 1 : file,
                line, what ? what : "", cc3_strerror(status));
  return status;
}
}  // namespace cc3

namespace cc3 {
static const char *kTraceNames[TR_NCLASS] = {"fp64_engine", "fp64_elementwise", "split_w_build",
                                             "split_omega", "split_elementwise", "output"};
void trace_begin(cc3_ctx *c, int cls, cudaStream_t s) {
  Tracer &T = c->trace;
  if (!T.on) return;
  auto &v = T.ev[cls];
  if ((int)v.size() < 2 * (T.used[cls] + 1)) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      v.push_back(e);
    }
  }
  cudaEventRecord(v[2 * T.used[cls]], s);
}
void trace_end(cc3_ctx *c, int cls, cudaStream_t s, double flop, double slice_flop) {
  Tracer &T = c->trace;
  if (!T.on) return;
  auto &v = T.ev[cls];
  if ((int)v.size() < 2 * (T.used[cls] + 1)) return;
  cudaEventRecord(v[2 * T.used[cls] + 1], s);
  T.used[cls]++;
  T.launches[cls]++;
  T.flop[cls] += flop;
  T.slice_flop[cls] += slice_flop;
}
void trace_reset(cc3_ctx *c) {
  Tracer &T = c->trace;
  for (int k = 0; k < TR_NCLASS; ++k) {
    T.used[k] = 0;
    T.launches[k] = 0;
    T.flop[k] = T.slice_flop[k] = T.ms[k] = 0.0;
  }
}
int trace_collect(cc3_ctx *c, cudaStream_t s) {
  Tracer &T = c->trace;
  if (!T.on) return CC3_OK;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, "trace sync");
  for (int k = 0; k < TR_NCLASS; ++k)
    for (int i = 0; i < T.used[k]; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, T.ev[k][2 * i], T.ev[k][2 * i + 1]) == cudaSuccess)
        T.ms[k] += ms;
    }
  return CC3_OK;
}
}  // namespace cc3

extern "C" {

const char *cc3_last_error(void) { return cc3::g_last_error; }

int cc3_ctx_set_tracing(cc3_ctx *c, int on) {
  if (!c) return CC3_ERR_ARG;
  c->trace.on = on != 0;
  return CC3_OK;
}

int cc3_ctx_trace(const cc3_ctx *c, cc3_trace *out) {
  if (!c || !out) return CC3_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  for (int k = 0; k < TR_NCLASS; ++k) {
    cc3_trace_entry &e = out->e[out->n++];
    std::snprintf(e.name, sizeof(e.name), "%s", kTraceNames[k]);
    e.launches = c->trace.launches[k];
    e.ms = c->trace.ms[k];
    e.flop = c->trace.flop[k];
    e.slice_flop = c->trace.slice_flop[k];
  }
  return CC3_OK;
}

const char *cc3_strerror(int status) {
  switch (status) {
    case CC3_OK: return "ok";
    case CC3_ERR_ARG: return "invalid argument";
    case CC3_ERR_OOM: return "out of memory";
    case CC3_ERR_CUDA: return "CUDA error";
    case CC3_ERR_TIMEOUT: return "bounded device wait timed out";
    case CC3_ERR_DENOM: return "vanishing or non-positive denominator";
    case CC3_ERR_BUSY: return "busy: request not admitted";
    case CC3_ERR_UNSUPPORTED: return "unsupported option";
    case CC3_ERR_NOT_FOUND: return "unknown ticket";
    case CC3_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

void cc3_ctx_destroy(cc3_ctx *c) {
  if (!c) return;
  CtxExtra *X = extra(c);
  if (X) {
    free_omega_plans(X->omega);
    if (X->escr) cudaFree(X->escr);
    if (X->om2tmp) cudaFree(X->om2tmp);
    delete X;
  }
  split_destroy(c);
  jacobian_destroy(c);
  for (int k = 0; k < TR_NCLASS; ++k)
    for (cudaEvent_t e : c->trace.ev[k]) cudaEventDestroy(e);
  double *bufs[] = {c->eps_o, c->eps_v, c->t2, c->vvvo, c->vvov, c->oovo, c->ooov,
                    c->ovov, c->F_ov, c->chol, c->vvoo, c->oooo, c->ws_w,
                    c->ws_tt, c->ws_tt2, c->omt, c->om1, c->Zv, c->Zo, c->R2,
                    c->hvvvo, c->hoovo, c->hF, c->rhot, c->rho1};
  for (double *p : bufs)
    if (p) cudaFree(p);
  if (c->status) cudaFree(c->status);
  if (c->omt_fx) cudaFree(c->omt_fx);
  if (c->om1_fx) cudaFree(c->om1_fx);
  delete c;
}

}  // extern "C"

// Context creation shared by the symmetric and the general entry points:
// g_oovo and g_vvov are null for symmetric integrals (oovo is then the
// transpose of ooov and the contractions read vvov through vvvo).
static int ctx_create_impl(cc3_ctx **out, int no, int nv, const double *eps_o,
                           const double *eps_v, const double *t2, const double *g_vvvo,
                           const double *g_oovo, const double *g_ooov, const double *g_ovov,
                           const double *g_vvov, const double *F_ov, const double *chol_L,
                           int naux, unsigned flags, void *cuda_stream) {
  if (!out) return CC3_ERR_ARG;
  *out = nullptr;
  if (no < 1 || nv < 1 || nv > 1024 || no > 256) return CC3_ERR_ARG;
  if (!eps_o || !eps_v || !t2 || !g_vvvo || !g_ooov || !g_ovov || !F_ov)
    return CC3_ERR_ARG;
  if ((g_oovo == nullptr) != (g_vvov == nullptr)) return CC3_ERR_ARG;
  if (naux < 0 || (naux > 0 && !chol_L)) return CC3_ERR_ARG;
  if (flags & ~(CC3_DEVICE_PTRS | CC3_DETERMINISTIC)) return CC3_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cc3_ctx *c = new (std::nothrow) cc3_ctx();
  if (!c) return CC3_ERR_OOM;
  c->ext = new (std::nothrow) CtxExtra();
  if (!c->ext) { delete c; return CC3_ERR_OOM; }
  c->no = no;
  c->nv = nv;
  c->naux = chol_L ? naux : 0;
  c->flags = flags;
  c->stream0 = s;
  cudaGetDevice(&c->device);
  const size_t nvvvo = (size_t)nv * nv * nv * no, nooov = (size_t)no * no * no * nv,
               novov = (size_t)no * nv * no * nv, nt2 = (size_t)no * no * nv * nv;
  const cudaMemcpyKind k = in_kind(c);
  int rc = CC3_OK;
#define ALLOC_COPY(dst, src, n)                                                \
  do {                                                                         \
    if ((rc = dalloc(&c->dst, (n))) != CC3_OK) goto fail;                      \
    if (cudaMemcpyAsync(c->dst, (src), sizeof(double) * (n), k, s) !=          \
        cudaSuccess) { rc = CC3_ERR_CUDA; goto fail; }                        \
  } while (0)
  ALLOC_COPY(eps_o, eps_o, (size_t)no);
  ALLOC_COPY(eps_v, eps_v, (size_t)nv);
  ALLOC_COPY(t2, t2, nt2);
  ALLOC_COPY(vvvo, g_vvvo, nvvvo);
  ALLOC_COPY(ooov, g_ooov, nooov);
  ALLOC_COPY(ovov, g_ovov, novov);
  if (g_vvov) {
    c->general = true;
    ALLOC_COPY(vvov, g_vvov, nvvvo);
    ALLOC_COPY(oovo, g_oovo, nooov);
  }
  ALLOC_COPY(F_ov, F_ov, (size_t)no * nv);
  if (c->naux > 0) {
    const size_t n = (size_t)no + nv;
    ALLOC_COPY(chol, chol_L, (size_t)naux * n * n);
  }
#undef ALLOC_COPY
  if (!c->general) {
    if ((rc = dalloc(&c->oovo, nooov)) != CC3_OK) goto fail;
    if ((rc = launch_transpose_ooov_to_oovo(c->ooov, c->oovo, no, nv, s)) != CC3_OK) goto fail;
  }
  if ((rc = dalloc(&c->omt, nt2)) != CC3_OK) goto fail;
  if ((rc = dalloc(&c->om1, (size_t)no * nv)) != CC3_OK) goto fail;
  if (flags & CC3_DETERMINISTIC) {
    if (cudaMalloc(&c->omt_fx, sizeof(unsigned long long) * 2 * nt2) != cudaSuccess ||
        cudaMalloc(&c->om1_fx, sizeof(unsigned long long) * 2 * (size_t)no * nv) != cudaSuccess) {
      rc = CC3_ERR_OOM;
      goto fail;
    }
  }
  if ((rc = dalloc(&extra(c)->escr, 257)) != CC3_OK) goto fail;
  if (cudaMalloc(&c->status, sizeof(int) * 4) != cudaSuccess) { rc = CC3_ERR_OOM; goto fail; }
  if (cudaMemsetAsync(c->status, 0, sizeof(int) * 4, s) != cudaSuccess) { rc = CC3_ERR_CUDA; goto fail; }
  default_triples(c);
  c->batch = choose_batch(c);
  if ((rc = alloc_workspace(c)) != CC3_OK) goto fail;
  {
    // orbital-energy sanity: every denominator eps^{abc}_{ijk} must be > 0
    std::vector<double> eo(no), ev(nv);
    if (cudaMemcpyAsync(eo.data(), c->eps_o, sizeof(double) * no, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(ev.data(), c->eps_v, sizeof(double) * nv, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { rc = CC3_ERR_CUDA; goto fail; }
    const double emin = 3.0 * *std::min_element(ev.begin(), ev.end()) -
                        3.0 * *std::max_element(eo.begin(), eo.end());
    if (!(emin > 0.0)) { rc = CC3_ERR_DENOM; goto fail; }
    c->eo_h = eo;
    c->ev_h = ev;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) { rc = CC3_ERR_CUDA; goto fail; }
  *out = c;
  return CC3_OK;
fail:
  cudaGetLastError();
  cc3_ctx_destroy(c);
  return rc;
}

extern "C" {

int cc3_ctx_create(cc3_ctx **out, int no, int nv, const double *eps_o,
                   const double *eps_v, const double *t2, const double *g_vvvo,
                   const double *g_ooov, const double *g_ovov,
                   const double *F_ov, const double *chol_L, int naux,
                   unsigned flags, void *cuda_stream) {
  return ctx_create_impl(out, no, nv, eps_o, eps_v, t2, g_vvvo, nullptr, g_ooov, g_ovov,
                         nullptr, F_ov, chol_L, naux, flags, cuda_stream);
}

int cc3_ctx_create_general(cc3_ctx **out, int no, int nv, const double *eps_o,
                           const double *eps_v, const double *t2, const double *g_vvvo,
                           const double *g_oovo, const double *g_ooov, const double *g_ovov,
                           const double *g_vvov, const double *F_ov, unsigned flags,
                           void *cuda_stream) {
  if (!g_oovo || !g_vvov) return CC3_ERR_ARG;
  return ctx_create_impl(out, no, nv, eps_o, eps_v, t2, g_vvvo, g_oovo, g_ooov, g_ovov, g_vvov,
                         F_ov, nullptr, 0, flags, cuda_stream);
}

int cc3_ctx_set_triples(cc3_ctx *c, int ntri, const int *ijk) {
  if (!c || ntri < 0) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  if (ntri == 0 || !ijk) {
    default_triples(c);
  } else {
    std::vector<int> v(ijk, ijk + 3 * (size_t)ntri);
    for (int t = 0; t < ntri; ++t) {
      const int i = v[3 * t], j = v[3 * t + 1], k = v[3 * t + 2];
      if (!(i < c->no && i >= j && j >= k && k >= 0)) return CC3_ERR_ARG;
    }
    c->tri_host = v;
    c->ntri = ntri;
  }
  const int nb = choose_batch(c);
  if (nb != c->batch) {
    c->batch = nb;
    TRY(alloc_workspace(c));
  }
  extra(c)->omega.valid = false;
  split_invalidate(c);
  c->prep_valid = false;
  return CC3_OK;
}

int cc3_cvs_triples(int no, int ncore, const int *core, int max, int *ijk) {
  if (no < 0 || ncore < 0 || ncore > no || (ncore > 0 && !core) || max < 0 ||
      (max > 0 && !ijk))
    return CC3_ERR_ARG;
  std::vector<char> is_core((size_t)no, 0);
  for (int u = 0; u < ncore; ++u) {
    if (core[u] < 0 || core[u] >= no || is_core[core[u]]) return CC3_ERR_ARG;
    is_core[core[u]] = 1;
  }
  long long n = 0;
  for (int i = 0; i < no; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k) {
        if (i == k) continue;  // i = j = k contributes nothing
        if (!is_core[i] && !is_core[j] && !is_core[k]) continue;
        if (n < max) {
          ijk[3 * n] = i;
          ijk[3 * n + 1] = j;
          ijk[3 * n + 2] = k;
        }
        ++n;
      }
  return n > 0x7fffffffLL ? CC3_ERR_ARG : (int)n;
}

int cc3_denominator_gap(int no, int nv, const double *eps_o, const double *eps_v, int ntri,
                        const int *ijk, double w, double *gap) {
  if (no < 1 || nv < 1 || !eps_o || !eps_v || !gap || ntri < 0 || (ntri > 0 && !ijk) ||
      !std::isfinite(w))
    return CC3_ERR_ARG;
  for (int t = 0; t < ntri; ++t) {
    const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
    if (!(i < no && i >= j && j >= k && k >= 0)) return CC3_ERR_ARG;
  }
  for (int p = 0; p < no; ++p)
    if (!std::isfinite(eps_o[p])) return CC3_ERR_ARG;
  for (int a = 0; a < nv; ++a)
    if (!std::isfinite(eps_v[a])) return CC3_ERR_ARG;
  *gap = denominator_gap(no, nv, eps_o, eps_v, ntri, ntri > 0 ? ijk : nullptr, w);
  return CC3_OK;
}

int cc3_ctx_counters(const cc3_ctx *c, cc3_counters *out) {
  if (!c || !out) return CC3_ERR_ARG;
  *out = c->counters;
  return CC3_OK;
}

int cc3_ctx_autotune(cc3_ctx *c, void *cuda_stream, int *ksteps_per_tile, int *ntile_w) {
  if (!c) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->ntri == 0) return CC3_OK;
  return split_autotune(c, (cudaStream_t)cuda_stream, ksteps_per_tile, ntile_w);
}

int cc3_ctx_get_tuning(cc3_ctx *c, int *ksteps_per_tile, int *ntile_w) {
  if (!c) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  return split_tuning(c, ksteps_per_tile, ntile_w);
}

int cc3_ctx_set_slices(cc3_ctx *c, int slices) {
  if (!c || slices < 3 || slices > 7) return CC3_ERR_ARG;
  c->slices = slices;
  split_invalidate(c);
  return CC3_OK;
}

// Weighted triple count: sum over the loop of the distinct permutations.
static long long weighted(const cc3_ctx *c) {
  long long w = 0;
  for (int t = 0; t < c->ntri; ++t) w += weight_of(&c->tri_host[3 * t]);
  return w;
}

static int finish_outputs(cc3_ctx *c, double *Omega1, double *Omega2,
                          double *E_T, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const size_t nt2 = (size_t)no * no * nv * nv;
  CtxExtra *X = extra(c);
  if (Omega2) {
    double *dst = Omega2;
    if (!(c->flags & CC3_DEVICE_PTRS)) {
      if (!X->om2tmp) TRY(dalloc(&X->om2tmp, nt2));
      dst = X->om2tmp;
    }
    TRY(launch_back_transform(c->omt, dst, no, nv, s));
    c->counters.launches++;
    if (dst != Omega2)
      CU(cudaMemcpyAsync(Omega2, dst, sizeof(double) * nt2, cudaMemcpyDeviceToHost, s));
  }
  if (Omega1)
    CU(cudaMemcpyAsync(Omega1, c->om1, sizeof(double) * no * nv, out_kind(c), s));
  if (E_T) {
    TRY(launch_energy(c->t2, c->omt, X->escr, no, nv, s));
    c->counters.launches += 2;
    CU(cudaMemcpyAsync(E_T, X->escr, sizeof(double), out_kind(c), s));
  }
  if (!(c->flags & CC3_DEVICE_PTRS)) CU(cudaStreamSynchronize(s));
  CU(cudaGetLastError());
  return CC3_OK;
}

static int omega_fp64(cc3_ctx *c, cudaStream_t s) {
  CtxExtra *X = extra(c);
  if (!X->omega.valid) TRY(build_omega_plans(c, s));
  PtrTable pt;
  fill_ptrs(c, &pt);
  const size_t nv3 = (size_t)c->nv * c->nv * c->nv;
  for (size_t b = 0; b < X->omega.ab.size(); ++b) {
    for (const DevPlan *d : {&X->omega.ab[b], &X->omega.c[b]}) {
      trace_begin(c, TR_FP64_ENGINE, s);
      TRY(launch_plan(*d, pt, s, &c->counters.launches));
      trace_end(c, TR_FP64_ENGINE, s, d->flop, 0.0);
    }
    trace_begin(c, TR_FP64_ELEM, s);
    TRY(launch_contravariant(c->ws_w, c->ws_tt, c->nv, X->omega.nslot[b], s));
    trace_end(c, TR_FP64_ELEM, s, 0.0, 0.0);
    c->counters.launches++;
    for (const DevPlan *d : {&X->omega.om[b], &X->omega.thin[b]}) {
      trace_begin(c, TR_FP64_ENGINE, s);
      TRY(launch_plan(*d, pt, s, &c->counters.launches));
      trace_end(c, TR_FP64_ENGINE, s, d->flop, 0.0);
    }
  }
  (void)nv3;
  c->counters.executed_flop = X->omega.executed;
  c->counters.slices = 0;
  return CC3_OK;
}

int cc3_omega_triples(cc3_ctx *c, cc3_prec prec, double *Omega1,
                      double *Omega2, double *E_T, void *cuda_stream) {
  if (!c) return CC3_ERR_ARG;
  if (prec != CC3_FP64 && prec != CC3_SPLIT_BF16 && prec != CC3_SPLIT_INT8)
    return CC3_ERR_ARG;
  if (prec == CC3_SPLIT_INT8) return CC3_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int no = c->no, nv = c->nv;
  const size_t nt2 = (size_t)no * no * nv * nv;
  c->counters = cc3_counters{};
  trace_reset(c);
  c->counters.nominal_flop = 4.0 * (double)nv * nv * nv * nv * (double)weighted(c);
  TRY(launch_zero(c->omt, nt2, s));
  TRY(launch_zero(c->om1, (size_t)no * nv, s));
  c->counters.launches += 2;
  if (c->omt_fx) {  // deterministic: the sums accumulate in 128-bit fixed point
    CU(cudaMemsetAsync(c->omt_fx, 0, sizeof(unsigned long long) * 2 * nt2, s));
    CU(cudaMemsetAsync(c->om1_fx, 0, sizeof(unsigned long long) * 2 * (size_t)no * nv, s));
  }
  if (prec == CC3_FP64) {
    TRY(omega_fp64(c, s));
  } else {
    TRY(split_omega(c, s));
  }
  if (c->omt_fx) {
    TRY(launch_fx_to_double(c->omt_fx, c->omt, nt2, s));
    TRY(launch_fx_to_double(c->om1_fx, c->om1, (size_t)no * nv, s));
    c->counters.launches += 2;
  }
  trace_begin(c, TR_OUTPUT, s);
  const int rc = finish_outputs(c, Omega1, Omega2, E_T, s);
  trace_end(c, TR_OUTPUT, s, 0.0, 0.0);
  if (rc != CC3_OK) return rc;
  return trace_collect(c, s);
}

}  // extern "C"
