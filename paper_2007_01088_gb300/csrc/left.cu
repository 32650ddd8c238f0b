// Left (transpose) CC3 Jacobian transformation, triples part (paper: the
// transpose-Jacobian paragraph of "Implementation"; the L3 amplitudes of
// Algorithm 3), FP64 path.
//
// The left transformation is the exact transpose of the right one
// (jacobian.cu) under the plain inner product over the elements of (R1, R2):
// sum L . rho(R) = sum sigma(L) . R.  With Lt2 the back-transform applied to L2
// (that map is its own transpose) and, per distinct permutation (p,q,r) of a
// loop triple, V the contravariant amplitudes viewed with x, y, z in the slots
// of p, q, r:
//   loop 1 (tau3):  Q[r][z] += sum_xy Lt2[p][q][x][y] V[x][y][z]
//   loop 2 (L3):    X_pqr[x][y][z] = L1[p][x] (qy|rz) + Lt2[p][q][x][y] F[r][z]
//                                  + (the W-build bracket with t2 -> Lt2)
//                   L3 = P X / (w - eps),  V = contravariant(L3)
//                   sigma2 += the residual's vvov and ooov contractions of V
//                   G[y][d][z][r] += sum_x V[x][y][z] t[p][q][x][d]
//                   H[l][q][z][r] += sum_xy V[x][y][z] t[p][l][x][y]
//   after the loops (the R1 dependence of the dressed integrals, transposed):
//     sigma1 += F^(Q) + Z~v . Lt2 - Z~o . Lt2  (Algorithm 2 intermediates)
//            - G . (ld|ck) - G . (bd|lk) + G . (bd|ce)   (vvvv via Cholesky)
//            - H . (ld|ck) + H . (lj|mk) - H . (lj|cd)
//     sigma2 <- (sigma2 + sigma2^{ji,ba}) / 2
// tau~3 is built once per batch of triples and shared by all vectors; the
// cost is (2 + 6 nvec) nv^4 per distinct permutation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
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

static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
__constant__ int kPerm6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                 {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};

// W[slot][c][a][b] += sum over the six terms of P of
//   L1[o0][x] (o1 y|o2 z) + Lt2[o0][o1][x][y] F[o2][z]
// with (o0,o1,o2) = (ijk[s0], ijk[s1], ijk[s2]), (x,y,z) = (v[s0], v[s1],
// v[s2]), v = (a, b, c): the outer products of the L3 numerator.
__global__ void left_outer_kernel(double *__restrict__ W, const int *__restrict__ tri,
                                  const double *__restrict__ L1,
                                  const double *__restrict__ Lt,
                                  const double *__restrict__ ovov,
                                  const double *__restrict__ F, int no, int nv) {
  const int slot = blockIdx.y;
  const int ijk[3] = {tri[3 * slot], tri[3 * slot + 1], tri[3 * slot + 2]};
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  double *Ws = W + slot * nv3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv3;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % nv), a = (int)((e / nv) % nv), c = (int)(e / nv2);
    const int v[3] = {a, b, c};
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int o0 = ijk[kPerm6[u][0]], o1 = ijk[kPerm6[u][1]], o2 = ijk[kPerm6[u][2]];
      const int x = v[kPerm6[u][0]], y = v[kPerm6[u][1]], z = v[kPerm6[u][2]];
      s += L1[(long long)o0 * nv + x] *
               ovov[(((long long)o1 * nv + y) * no + o2) * nv + z] +
           Lt[(((long long)o0 * no + o1) * nv + x) * nv + y] * F[(long long)o2 * nv + z];
    }
    Ws[e] += s;
  }
}

// out[i][j][a][b] = (in[i][j][a][b] + in[j][i][b][a]) / 2
__global__ void pair_symmetrize_kernel(const double *__restrict__ in, double *__restrict__ out,
                                       int no, int nv) {
  const long long nv2 = (long long)nv * nv, n = (long long)no * no * nv2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % nv), a = (int)((e / nv) % nv);
    const int j = (int)((e / nv2) % no), i = (int)(e / (nv2 * no));
    out[e] = 0.5 * (in[e] + in[((long long)j * no + i) * nv2 + (long long)b * nv + a]);
  }
}

int grid_for(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, 8192LL)); }

struct Bufs {
  std::vector<void *> p;
  ~Bufs() {
    for (void *x : p)
      if (x) cudaFree(x);
  }
  template <class T>
  int get(T **out, size_t n) {
    *out = nullptr;
    if (cudaMalloc(out, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
      cudaGetLastError();
      return CC3_FAIL(CC3_ERR_OOM, "left Jacobian workspace");
    }
    p.push_back(*out);
    return CC3_OK;
  }
};

// Per-permutation jobs of the L3 loop on the contravariant amplitudes in
// slot `slot` of B_WS_TTR ([a][b][c] per slot): G, H (rows as in the header)
void plan_left_gh(Plan &pg, Plan &ph, int no, int nv, const int ijk[3], int slot) {
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long st[3] = {nv2, nv, 1};
  int maps[6][3], np = 0;
  for (int u = 0; u < 6 && !(ijk[0] == ijk[1] && ijk[1] == ijk[2]); ++u) {
    bool dup = false;
    for (int w = 0; w < np; ++w)
      if (ijk[maps[w][0]] == ijk[PERM6[u][0]] && ijk[maps[w][1]] == ijk[PERM6[u][1]] &&
          ijk[maps[w][2]] == ijk[PERM6[u][2]])
        dup = true;
    if (dup) continue;
    for (int k = 0; k < 3; ++k) maps[np][k] = PERM6[u][k];
    ++np;
  }
  const long long tt0 = slot * nv3;
  for (int u = 0; u < np; ++u) {
    const int *m = maps[u];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    // G[y][d][z][r] += sum_x V[x][y][z] t[p][q][x][d]: rows (y, z), cols d, K = x
    int jb = new_job(pg, 0, (int)nv2, nv, nv, 1, 1, EPI_ATOMIC);
    add_term(pg, jb, with_m2(op(B_WS_TTR, tt0, st[m[2]], st[m[0]]), nv, st[m[1]]),
             op(B_T2, ((long long)p * no + q) * nv2, 1, nv), nv);
    OutD o = out(B_G, r, no, (long long)nv * no);
    o.m_in = nv;
    o.sm1 = nv2 * no;
    pg.jobs[jb].C = o;
    pg.jobs[jb].Ct = o;
    // H[l][q][z][r] += sum_xy V[x][y][z] t[p][l][x][y]: rows z, cols l, K = (x, y)
    jb = new_job(ph, 1, nv, no, no, 1, 1, EPI_ATOMIC);
    add_term(ph, jb, with_k2(op(B_WS_TTR, tt0, st[m[2]], st[m[1]]), nv, st[m[0]]),
             op(B_T2, (long long)p * no * nv2, nv2, 1), (int)nv2);
    o = out(B_H, (long long)q * nv * no + r, no, (long long)no * nv * no);
    ph.jobs[jb].C = o;
    ph.jobs[jb].Ct = o;
  }
}

}  // namespace

// Q[r][z] += sum_xy Lt2[p][q][x][y] V[x][y][z] for every distinct permutation
// (V: tau~3 in slot `slot` of B_WS_TT)
void plan_left_q(Plan &P, int no, int nv, const int ijk[3], int slot) {
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long st[3] = {nv2, nv, 1};
  int seen[6][3], ns = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int u = 0; u < 6; ++u) {
    const int *m = PERM6[u];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int w = 0; w < ns; ++w)
      if (seen[w][0] == p && seen[w][1] == q && seen[w][2] == r) dup = true;
    if (dup) continue;
    seen[ns][0] = p;
    seen[ns][1] = q;
    seen[ns][2] = r;
    ++ns;
    const int jb = new_job(P, 1, nv, 1, 1, 1, 1, EPI_ATOMIC);
    add_term(P, jb, with_k2(op(B_WS_TT, slot * nv3, st[m[2]], st[m[1]]), nv, st[m[0]]),
             op(B_LT, ((long long)p * no + q) * nv2, 0, 1), (int)nv2);
    const OutD o = out(B_Q, (long long)r * nv, 1, 0);
    P.jobs[jb].C = o;
    P.jobs[jb].Ct = o;
  }
}

// Covariant L3 = P X / (w - eps) of the triples [t0, t1) into wsW (slot layout
// [c][a][b], as the W build writes it) and its contravariant form into wsT
// ([a][b][c]).  pt: B_LT = ltd (the back-transformed L2), B_WS_WR = wsW;
// tri: device room for 3 (t1 - t0) ints.
int left_l3_batch(cc3_ctx *c, const PtrTable &pt, int t0, int t1, double w, const double *L1d,
                  const double *ltd, int *tri, double *wsW, double *wsT, cudaStream_t s) {
  const int no = c->no, nv = c->nv, ns = t1 - t0;
  const long long nv3 = (long long)nv * nv * nv;
  const TermSet set{B_LT, B_VVVO, B_OOVO};
  Plan pab, pc;
  for (int t = t0; t < t1; ++t) {
    const int *ijk = &c->tri_host[3 * t];
    const double e = c->eo_h[ijk[0]] + c->eo_h[ijk[1]] + c->eo_h[ijk[2]];
    plan_w_build(pab, no, nv, ijk, t - t0, B_WS_WR, &set, 1, 0.0, 0.0, 0);
    plan_w_build(pc, no, nv, ijk, t - t0, B_WS_WR, &set, 1, w, e, 1);
  }
  CU(cudaMemcpyAsync(tri, &c->tri_host[3 * t0], sizeof(int) * 3 * ns, cudaMemcpyHostToDevice, s));
  TRY(jac_run_plan(c, pab, 0, pt, s));
  left_outer_kernel<<<dim3(grid_for(nv3 / 4), ns), 256, 0, s>>>(wsW, tri, L1d, ltd, c->ovov,
                                                                 c->F_ov, no, nv);
  CU(cudaGetLastError());
  c->counters.launches++;
  TRY(jac_run_plan(c, pc, 0, pt, s));
  trace_begin(c, TR_FP64_ELEM, s);
  TRY(launch_contravariant(wsW, wsT, nv, ns, s));
  trace_end(c, TR_FP64_ELEM, s, 0.0, 0.0);
  c->counters.launches++;
  return CC3_OK;
}

namespace {

// sigma1 terms outside the loops (rows and columns as in the header); with
// chol_done the Cholesky product N = L . G is already in B_MJ
int left_singles(cc3_ctx *c, const PtrTable &pt, cudaStream_t s, bool chol_done = false) {
  const int no = c->no, nv = c->nv, n = no + nv, naux = c->naux;
  const long long nv2 = (long long)nv * nv, nvo = (long long)nv * no, n2 = (long long)n * n;
  const long long ovl = (long long)nv * no * nv;  // stride of the first ovov index
  const long long no3 = (long long)no * no * no;
  Plan thin, wide, chol1;
  const OutD s1 = [&] {
    OutD o = out(B_S1, 0, 1, nv);  // sigma1[col][row]
    return o;
  }();
  int jb;
  // F^(Q): sum_kc Q[k][c] [2 (kc|ld) - (kd|lc)] (the symmetric matrix of F^)
  jb = new_job(thin, 1, no * nv, 1, 0, 1, 1, EPI_ATOMIC);
  {
    const Opnd Bt = with_k2(op(B_Q, 0, 0, 1), nv, nv);
    const Opnd Aa = with_k2(with_m2(op(B_OVOV, 0, nvo, 1), nv, ovl), nv, nv);
    const Opnd Ab = with_k2(with_m2(op(B_OVOV, 0, 1, nvo, 0, 1), nv, ovl), nv, nv);
    add_term(thin, jb, Aa, Bt, no * nv, &Bt);
    add_term(thin, jb, Aa, Bt, no * nv, &Bt);
    add_term(thin, jb, Ab, Bt, no * nv, &Bt);
    OutD o = out(B_S1, 0, 1, 0);
    o.m_in = nv;
    o.sm1 = nv;
    thin.jobs[jb].C = o;
    thin.jobs[jb].Ct = o;
  }
  // Z~v: + sum_{p,a,b} Lt2[p][l][a][b] Z~v[a][b][p][d]   (batch p)
  jb = new_job(thin, 1, nv, no, no, no, 1, EPI_ATOMIC);
  add_term(thin, jb, op(B_ZV, 0, 1, nvo, nv), op(B_LT, 0, nv2, 1, (long long)no * nv2), (int)nv2);
  thin.jobs[jb].C = s1;
  thin.jobs[jb].Ct = s1;
  // Z~o: - sum_{p,q,a} Lt2[p][q][a][d] Z~o[a][q][p][l]   (batch p)
  jb = new_job(thin, 1, nv, no, no, no, 1, EPI_ATOMIC);
  add_term(thin, jb, with_k2(op(B_LT, 0, 1, nv, (long long)no * nv2, 1), nv, nv2),
           with_k2(op(B_ZO, 0, 1, no3, no), nv, (long long)no * no), no * nv);
  thin.jobs[jb].C = s1;
  thin.jobs[jb].Ct = s1;
  // G: - sum_{d,c,k} G[b][d][c][k] (ld|ck)   (batch d; rows b, cols l)
  jb = new_job(thin, 1, nv, no, no, nv, 1, EPI_ATOMIC);
  add_term(thin, jb, op(B_G, 0, nv2 * no, 1, nvo, 1),
           with_k2(op(B_OVOV, 0, ovl, nv, nvo), no, 1), (int)nvo);
  thin.jobs[jb].C = s1;
  thin.jobs[jb].Ct = s1;
  // G: - sum_{b,d,k} G[b][d][c][k] (lk|bd)   (batch b; rows c, cols l)
  jb = new_job(thin, 1, nv, no, no, nv, 1, EPI_ATOMIC);
  add_term(thin, jb, with_k2(op(B_G, 0, no, 1, nv2 * no, 1), no, nvo),
           with_k2(op(B_VVOO, 0, (long long)no * nv2, nv2, nv), no, 1), (int)nvo);
  thin.jobs[jb].C = s1;
  thin.jobs[jb].Ct = s1;
  // G, Cholesky term: N[J][(c,k)] = sum_bd L^J_bd G[b][d][c][k] (store), then
  // sigma1[k][e] += sum_{J,c} N[J][c][k] L^J_ce
  jb = new_job(wide, 0, naux, (int)nvo, (int)nvo, 1, 1, EPI_STORE);
  add_term(wide, jb, with_k2(op(B_CHOL, (long long)no * n + no, n2, 1), nv, n),
           op(B_G, 0, 1, nvo), (int)nv2);
  {
    OutD o = out(B_MJ, 0, nvo, 1);
    wide.jobs[jb].C = o;
    wide.jobs[jb].Ct = o;
  }
  jb = new_job(chol1, 1, nv, no, no, 1, 1, EPI_ATOMIC);
  add_term(chol1, jb, with_k2(op(B_CHOL, (long long)no * n + no, 1, n), nv, n2),
           with_k2(op(B_MJ, 0, 1, no), nv, nvo), naux * nv);
  chol1.jobs[jb].C = s1;
  chol1.jobs[jb].Ct = s1;
  // H: - sum_{l,c,k} H[l][j][c][k] (ld|ck)   (batch l; rows d, cols j)
  jb = new_job(chol1, 1, nv, no, no, no, 1, EPI_ATOMIC);
  add_term(chol1, jb, with_k2(op(B_OVOV, 0, nvo, nv, ovl, 1), no, 1),
           op(B_H, 0, nvo, 1, (long long)no * nvo), (int)nvo);
  chol1.jobs[jb].C = s1;
  chol1.jobs[jb].Ct = s1;
  // H: + sum_{l,j,k} H[l][j][c][k] (lj|mk)   (batch l; rows c, cols m)
  jb = new_job(chol1, 1, nv, no, no, no, 1, EPI_ATOMIC);
  add_term(chol1, jb, with_k2(op(B_H, 0, no, 1, (long long)no * nvo), no, nvo),
           with_k2(op(B_OOOO, 0, no, 1, no3), no, (long long)no * no), no * no);
  chol1.jobs[jb].C = s1;
  chol1.jobs[jb].Ct = s1;
  // H: - sum_{l,j,c} H[l][j][c][k] (lj|cd)   (batch (l,j); rows d, cols k)
  jb = new_job(chol1, 1, nv, no, no, no * no, 1, EPI_ATOMIC);
  add_term(chol1, jb, op(B_VVOO, 0, 1, nv, nv2, 1), op(B_H, 0, 1, no, nvo), nv);
  chol1.jobs[jb].C = s1;
  chol1.jobs[jb].Ct = s1;
  TRY(jac_run_plan(c, thin, 1, pt, s));
  if (!chol_done) TRY(jac_run_plan(c, wide, 0, pt, s));
  TRY(jac_run_plan(c, chol1, 1, pt, s));
  return CC3_OK;
}

int left_fp64(cc3_ctx *c, int nvec, const double *w, const double *L1d, const double *L2d,
              double *s1d, double *s2d, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv;
  TRY(jac_prep_fp64(c, s));  // (lj|mk), (lj|cd) and the Algorithm 2 intermediates
  Bufs B;
  double *lt = nullptr, *s2raw = nullptr, *Q = nullptr, *G = nullptr, *H = nullptr,
         *N = nullptr, *wsW = nullptr, *wsT = nullptr;
  int *tri = nullptr;
  TRY(B.get(&lt, nt2 * nvec));
  TRY(B.get(&s2raw, nt2));
  TRY(B.get(&Q, n1 * nvec));
  TRY(B.get(&G, (size_t)nv3 * no));
  TRY(B.get(&H, (size_t)no * no * nv * no));
  TRY(B.get(&N, (size_t)c->naux * nv * no));
  TRY(B.get(&wsW, (size_t)nv3 * c->batch));
  TRY(B.get(&wsT, (size_t)nv3 * c->batch));
  TRY(B.get(&tri, 3 * (size_t)c->batch));
  TRY(launch_zero(Q, n1 * nvec, s));
  for (int v = 0; v < nvec; ++v) TRY(launch_back_transform(L2d + v * nt2, lt + v * nt2, no, nv, s));
  PtrTable base;
  jac_fill_ptrs(c, &base);
  base.p[B_G] = G;
  base.p[B_H] = H;
  base.p[B_MJ] = N;
  base.p[B_WS_WR] = wsW;
  base.p[B_WS_TTR] = wsT;
  auto vec_ptrs = [&](int v) {
    PtrTable pt = base;
    pt.p[B_LT] = lt + v * nt2;
    pt.p[B_Q] = Q + v * n1;
    pt.p[B_S1] = s1d + v * n1;
    pt.p[B_S2] = s2raw;
    return pt;
  };
  // loop 1: tau~3 per batch, contracted with every vector's Lt2 into Q
  for (int t0 = 0; t0 < c->ntri; t0 += c->batch) {
    const int t1 = std::min(c->ntri, t0 + c->batch);
    TRY(jac_tau_batch(c, t0, t1, s));
    Plan pq;
    for (int t = t0; t < t1; ++t) plan_left_q(pq, no, nv, &c->tri_host[3 * t], t - t0);
    for (int v = 0; v < nvec; ++v) TRY(jac_run_plan(c, pq, 1, vec_ptrs(v), s));
  }
  // loop 2, vector by vector: L3, its contravariant form, its contractions
  for (int v = 0; v < nvec; ++v) {
    const PtrTable pt = vec_ptrs(v);
    TRY(launch_zero(s1d + v * n1, n1, s));
    TRY(launch_zero(s2raw, nt2, s));
    TRY(launch_zero(G, (size_t)nv3 * no, s));
    TRY(launch_zero(H, (size_t)no * no * nv * no, s));
    for (int t0 = 0; t0 < c->ntri; t0 += c->batch) {
      const int t1 = std::min(c->ntri, t0 + c->batch);
      Plan pom, pth, pg, ph;
      for (int t = t0; t < t1; ++t) {
        const int *ijk = &c->tri_host[3 * t];
        // sigma2: the residual's vvov and ooov contractions, no tail columns
        plan_omega_contractions(pom, no, nv, ijk, t - t0, B_WS_TTR, B_OVOV, B_FOV, B_OOOV, true,
                                B_VVVO, B_S2, B_S1, 1, 1 | 8);
        plan_omega_contractions(pth, no, nv, ijk, t - t0, B_WS_TTR, B_OVOV, B_FOV, B_OOOV, true,
                                B_VVVO, B_S2, B_S1, 1, 2 | 8);
        plan_left_gh(pg, ph, no, nv, ijk, t - t0);
      }
      TRY(left_l3_batch(c, pt, t0, t1, w[v], L1d + v * n1, lt + v * nt2, tri, wsW, wsT, s));
      TRY(jac_run_plan(c, pom, 0, pt, s));
      TRY(jac_run_plan(c, pth, 1, pt, s));
      TRY(jac_run_plan(c, pg, 0, pt, s));
      TRY(jac_run_plan(c, ph, 1, pt, s));
    }
    TRY(left_singles(c, pt, s));
    pair_symmetrize_kernel<<<grid_for((long long)nt2), 256, 0, s>>>(s2raw, s2d + v * nt2, no, nv);
    CU(cudaGetLastError());
    c->counters.launches++;
  }
  CU(cudaStreamSynchronize(s));
  return CC3_OK;
}

}  // namespace

// sigma1 from Q, G, H, Lt2 and the cached Algorithm 2 intermediates (pt's
// B_Q, B_G, B_H, B_LT, B_ZV, B_ZO; output B_S1), then sigma2 = the pair-
// symmetric part of s2raw.  chol_done: B_MJ already holds N[J][(c,k)] =
// sum_bd L^J_bd G[b][d][c][k].
int left_finish(cc3_ctx *c, const PtrTable &pt, const double *s2raw, double *s2d,
                cudaStream_t s, bool chol_done) {
  TRY(left_singles(c, pt, s, chol_done));
  const long long nt2 = (long long)c->no * c->no * c->nv * c->nv;
  pair_symmetrize_kernel<<<grid_for(nt2), 256, 0, s>>>(s2raw, s2d, c->no, c->nv);
  CU(cudaGetLastError());
  c->counters.launches++;
  return CC3_OK;
}
}  // namespace cc3

extern "C" int cc3_left_jacobian_triples(cc3_ctx *c, cc3_prec prec, int nvec,
                                         const double *omega, const double *L1,
                                         const double *L2, double *sigma1, double *sigma2,
                                         void *cuda_stream) {
  using namespace cc3;
  if (!c || nvec < 1 || !omega || !L1 || !L2 || !sigma1 || !sigma2) return CC3_ERR_ARG;
  if (c->general)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "the Jacobian needs symmetric integrals");
  if (c->naux < 1 || !c->chol)
    return CC3_FAIL(CC3_ERR_ARG, "the Jacobian needs the Cholesky vectors (chol_L)");
  if (prec == CC3_SPLIT_INT8)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "no INT8 slice path");
  if (c->flags & CC3_DETERMINISTIC)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "deterministic reductions cover the residual only");
  if (prec != CC3_FP64 && prec != CC3_SPLIT_BF16) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  for (int v = 0; v < nvec; ++v) {
    if (!std::isfinite(omega[v])) return CC3_FAIL(CC3_ERR_ARG, "non-finite frequency");
    bool seen = false;
    for (int u = 0; u < v; ++u) seen = seen || omega[u] == omega[v];
    if (seen || c->ntri == 0) continue;
    if (denominator_gap(c->no, c->nv, c->eo_h.data(), c->ev_h.data(), c->ntri,
                        c->tri_host.data(), omega[v]) < CC3_DENOM_MIN)
      return CC3_FAIL(CC3_ERR_DENOM, "a frequency lies within CC3_DENOM_MIN of a triples "
                                     "denominator");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int no = c->no, nv = c->nv;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv;
  long long wsum = 0;
  for (int t = 0; t < c->ntri; ++t) {
    const int *x = &c->tri_host[3 * t];
    wsum += (x[0] == x[1] && x[1] == x[2]) ? 0 : ((x[0] != x[1] && x[1] != x[2]) ? 6 : 3);
  }
  c->counters = cc3_counters{};
  trace_reset(c);
  c->counters.nominal_flop = 8.0 * (double)nv * nv * nv * nv * (double)wsum * nvec;
  const bool dev = (c->flags & CC3_DEVICE_PTRS) != 0;
  double *dL1 = const_cast<double *>(L1), *dL2 = const_cast<double *>(L2), *ds1 = sigma1,
         *ds2 = sigma2;
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
    if (!mk(&dL1, n1 * nvec) || !mk(&dL2, nt2 * nvec) || !mk(&ds1, n1 * nvec) ||
        !mk(&ds2, nt2 * nvec))
      rc = CC3_FAIL(CC3_ERR_OOM, "left Jacobian staging");
    if (rc == CC3_OK &&
        (cudaMemcpyAsync(dL1, L1, sizeof(double) * n1 * nvec, cudaMemcpyHostToDevice, s) !=
             cudaSuccess ||
         cudaMemcpyAsync(dL2, L2, sizeof(double) * nt2 * nvec, cudaMemcpyHostToDevice, s) !=
             cudaSuccess))
      rc = CC3_FAIL(CC3_ERR_CUDA, "left Jacobian upload");
  }
  if (rc == CC3_OK) {
    if (c->ntri == 0) {
      rc = launch_zero(ds1, n1 * nvec, s);
      if (rc == CC3_OK) rc = launch_zero(ds2, nt2 * nvec, s);
    } else if (prec == CC3_SPLIT_BF16) {
      rc = split_left_jacobian(c, nvec, omega, dL1, dL2, ds1, ds2, s);
    } else {
      rc = left_fp64(c, nvec, omega, dL1, dL2, ds1, ds2, s);
    }
  }
  if (rc == CC3_OK && !dev) {
    if (cudaMemcpyAsync(sigma1, ds1, sizeof(double) * n1 * nvec, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(sigma2, ds2, sizeof(double) * nt2 * nvec, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = CC3_FAIL(CC3_ERR_CUDA, "left Jacobian download");
  }
  cudaStreamSynchronize(s);
  for (double *p : tmp) cudaFree(p);
  if (rc == CC3_OK) rc = trace_collect(c, s);
  return rc;
}
