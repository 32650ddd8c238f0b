// cc3_omega_triples_noalloc: the FP64 triples residual for small problems with
// every piece of scratch memory taken from one file-scope device array, for
// callers that cannot allocate device memory.
//
// Who needs this: code that runs inside a host framework which owns the GPU
// memory pool and forbids other allocations (a fixed-budget embedding, a
// plugin with a pre-reserved heap) can still call the triples residual as long
// as it passes its own input and output buffers.  The call reads the orbital
// energies back and synchronises its stream, so it is not capturable into a
// CUDA graph and must not overlap a global-mode capture on another thread.
//
// The scratch array below is part of the library image: every GPU that loads
// libcc3 holds it (16 MiB) until the process exits.  Its device address is
// looked up once per device (cudaGetSymbolAddress with that device current) on
// the first call, and again only if that device's context has changed since
// (after a cudaDeviceReset the module is loaded anew and the old address is
// stale).  All calls share the array, so calls that overlap on the GPU race;
// the contents left by the previous call are not relied on (the accumulators
// are cleared at the start of each call).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "cc3_internal.h"

namespace {

constexpr size_t kScratchDoubles = 2u << 20;  // 16 MiB
constexpr int kMaxNo = 12, kMaxNv = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
struct ScratchSlot {
  CUcontext ctx = nullptr;  // the device context the address belongs to
  double *ptr = nullptr;
};
ScratchSlot g_slot[64];

// The calling thread's current driver context (the runtime's primary context
// of the current device once it is initialised), through the runtime's
// driver entry point so that the library does not link the driver library.
CUcontext current_context() {
  using GetCurrent = CUresult (*)(CUcontext *);
  static GetCurrent fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCurrent>(f);
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array for the current device: set up on the
// first call per device, and again when the device's context changed.
int scratch_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return CC3_FAIL(CC3_ERR_CUDA, "no current device");
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchSlot &S = g_slot[dev];
  CUcontext now = current_context();
  if (!S.ptr || !now || now != S.ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e));
    S.ptr = static_cast<double *>(p);
    S.ctx = current_context();  // the lookup made the device's context current
  }
  *out = S.ptr;
  return CC3_OK;
}

size_t align_doubles(size_t n) { return (n + 31) / 32 * 32; }  // 256-byte steps

}  // namespace

extern "C" int cc3_omega_triples_noalloc(int no, int nv, const double *eps_o,
                                         const double *eps_v, const double *t2,
                                         const double *g_vvvo, const double *g_ooov,
                                         const double *g_ovov, const double *F_ov,
                                         double *Omega1, double *Omega2, double *E_T,
                                         void *cuda_stream) {
  using namespace cc3;
  if (no < 1 || nv < 1) return CC3_FAIL(CC3_ERR_ARG, "sizes");
  if (no > kMaxNo || nv > kMaxNv)
    return CC3_FAIL(CC3_ERR_ARG, "problem larger than the no-allocation limit (no <= 12, nv <= 64)");
  if (!eps_o || !eps_v || !t2 || !g_vvvo || !g_ooov || !g_ovov || !F_ov)
    return CC3_FAIL(CC3_ERR_ARG, "null input");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double *base = nullptr;
  {
    const int rc = scratch_for_current_device(&base);
    if (rc != CC3_OK) return rc;
  }
  const size_t nv3 = (size_t)nv * nv * nv, nt2 = (size_t)no * no * nv * nv;
  const size_t n_oovo = (size_t)no * no * no * nv;

  // triples i >= j >= k (not all equal), host plans for one triple in flight
  std::vector<int> tri;
  for (int i = 0; i < no; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k)
        if (!(i == j && j == k)) {
          tri.push_back(i);
          tri.push_back(j);
          tri.push_back(k);
        }
  const int ntri = (int)(tri.size() / 3);
  std::vector<double> eo(no), ev(nv);
  if (cudaMemcpyAsync(eo.data(), eps_o, sizeof(double) * no, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(ev.data(), eps_v, sizeof(double) * nv, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CC3_FAIL(CC3_ERR_CUDA, "reading the orbital energies");
  // every denominator eps^{abc}_{ijk} must be > 0 (the rule of cc3_ctx_create)
  if (!(3.0 * *std::min_element(ev.begin(), ev.end()) -
            3.0 * *std::max_element(eo.begin(), eo.end()) > 0.0))
    return CC3_FAIL(CC3_ERR_DENOM, "a triples denominator could be <= 0");
  const TermSet set{B_T2, B_VVVO, B_OOVO};
  Plan P[4];  // AB, C, residual (64x64 tiles), residual (thin tiles); all triples
  std::vector<int> j0[4];
  for (int t = 0; t < ntri; ++t) {
    const int *ijk = &tri[3 * t];
    const double e = eo[ijk[0]] + eo[ijk[1]] + eo[ijk[2]];
    for (int ph = 0; ph < 4; ++ph) j0[ph].push_back((int)P[ph].jobs.size());
    plan_w_build(P[0], no, nv, ijk, 0, B_WS_W, &set, 1, 0.0, e, 0);
    plan_w_build(P[1], no, nv, ijk, 0, B_WS_W, &set, 1, 0.0, e, 1);
    plan_omega_contractions(P[2], no, nv, ijk, 0, B_WS_TT, B_OVOV, B_FOV, B_OOOV, true, B_VVVO,
                            B_OMT, B_OM1, 2, 1);
    plan_omega_contractions(P[3], no, nv, ijk, 0, B_WS_TT, B_OVOV, B_FOV, B_OOOV, true, B_VVVO,
                            B_OMT, B_OM1, 1, 2);
  }
  for (int ph = 0; ph < 4; ++ph) j0[ph].push_back((int)P[ph].jobs.size());
  // every triple's jobs restart their tile numbering at 0 (one launch per triple)
  for (int ph = 0; ph < 4; ++ph)
    for (int t = 0; t < ntri; ++t) {
      const long long first = P[ph].jobs[j0[ph][t]].tile_base;
      for (int j = j0[ph][t]; j < j0[ph][t + 1]; ++j) P[ph].jobs[j].tile_base -= first;
    }

  // carve the scratch array
  size_t off = 0;
  auto take = [&](size_t n) {
    double *p = base + off;
    off += align_doubles(n);
    return p;
  };
  double *oovo = take(n_oovo), *ws_w = take(nv3), *ws_tt = take(nv3), *omt = take(nt2),
         *om1 = take((size_t)no * nv), *escr = take(257), *om2tmp = nullptr;
  size_t tbl_bytes[4][2];
  Job *jobs_dev[4];
  Term *terms_dev[4];
  for (int ph = 0; ph < 4; ++ph) {
    tbl_bytes[ph][0] = sizeof(Job) * P[ph].jobs.size();
    tbl_bytes[ph][1] = sizeof(Term) * P[ph].terms.size();
    jobs_dev[ph] = reinterpret_cast<Job *>(take((tbl_bytes[ph][0] + 7) / 8));
    terms_dev[ph] = reinterpret_cast<Term *>(take((tbl_bytes[ph][1] + 7) / 8));
  }
  if (!Omega2) om2tmp = nullptr;
  if (off > kScratchDoubles)
    return CC3_FAIL(CC3_ERR_ARG, "problem does not fit the no-allocation scratch (16 MiB)");
  for (int ph = 0; ph < 4; ++ph) {
    if (tbl_bytes[ph][0] &&
        cudaMemcpyAsync(jobs_dev[ph], P[ph].jobs.data(), tbl_bytes[ph][0],
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return CC3_FAIL(CC3_ERR_CUDA, "job table upload");
    if (tbl_bytes[ph][1] &&
        cudaMemcpyAsync(terms_dev[ph], P[ph].terms.data(), tbl_bytes[ph][1],
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return CC3_FAIL(CC3_ERR_CUDA, "term table upload");
  }
  // the host tables must stay alive until the copies have landed
  if (cudaStreamSynchronize(s) != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, "table upload");

  PtrTable pt;
  std::memset(&pt, 0, sizeof(pt));
  pt.p[B_T2] = const_cast<double *>(t2);
  pt.p[B_VVVO] = const_cast<double *>(g_vvvo);
  pt.p[B_OOVO] = oovo;
  pt.p[B_OOOV] = const_cast<double *>(g_ooov);
  pt.p[B_OVOV] = const_cast<double *>(g_ovov);
  pt.p[B_FOV] = const_cast<double *>(F_ov);
  pt.p[B_EPSV] = const_cast<double *>(eps_v);
  pt.p[B_EPSO] = const_cast<double *>(eps_o);
  pt.p[B_WS_W] = ws_w;
  pt.p[B_WS_TT] = ws_tt;
  pt.p[B_OMT] = omt;
  pt.p[B_OM1] = om1;
  pt.p[B_SCRATCH] = omt;

  int rc = launch_transpose_ooov_to_oovo(g_ooov, oovo, no, nv, s);
  if (rc == CC3_OK) rc = launch_zero(omt, nt2, s);
  if (rc == CC3_OK) rc = launch_zero(om1, (size_t)no * nv, s);
  for (int t = 0; t < ntri && rc == CC3_OK; ++t) {
    for (int ph = 0; ph < 4 && rc == CC3_OK; ++ph) {
      DevPlan d;
      d.jobs = jobs_dev[ph] + j0[ph][t];
      d.terms = terms_dev[ph];
      d.njobs = j0[ph][t + 1] - j0[ph][t];
      const Job &last = P[ph].jobs[j0[ph][t + 1] - 1];
      d.tiles = last.tile_base +
                (long long)last.batch * last.tiles_m * last.tiles_n * last.ksplit;
      d.tile_kind = ph == 3 ? 1 : 0;
      rc = launch_plan(d, pt, s, nullptr);
      if (ph == 1 && rc == CC3_OK) rc = launch_contravariant(ws_w, ws_tt, nv, 1, s);
    }
  }
  if (rc == CC3_OK && Omega2) rc = launch_back_transform(omt, Omega2, no, nv, s);
  if (rc == CC3_OK && Omega1 &&
      cudaMemcpyAsync(Omega1, om1, sizeof(double) * no * nv, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    rc = CC3_FAIL(CC3_ERR_CUDA, "Omega1 copy");
  if (rc == CC3_OK && E_T) {
    rc = launch_energy(t2, omt, escr, no, nv, s);
    if (rc == CC3_OK &&
        cudaMemcpyAsync(E_T, escr, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = CC3_FAIL(CC3_ERR_CUDA, "E_T copy");
  }
  (void)om2tmp;
  return rc;
}
