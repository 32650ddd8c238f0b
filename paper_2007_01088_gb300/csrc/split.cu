// Split-precision path of the CC3 triples residual (paper, Algorithm 1) on the
// tensor cores: staging of BF16 slice arrays, job plans and the
// per-batch launch sequence.
//
// Layouts (bf16, every array K-blocked as [slab][K/16][row group][slice][8 x 16]
// so that the slices of each 16 x R tile read by the tensor cores are one
// contiguous block; K zero padded to a multiple of 16; vp = nv rounded up,
// op = no rounded up):
//   T2S[(p,q)][x][d]  = t^{xd}_{pq}          T2C[(p,y)][x][l] = t^{xy}_{pl}
//   T2R[(p,x)][y][l]  = t^{xy}_{pl}          OS[(q,r)][z][l]  = (lq|zr)
//   XS[(r,z)][y][d]   = (yd|zr)              YS[(r,y)][z][d]  = (yd|zr)
//   Zg[r][d][(u,w)]   = (ud|wr)              Zh[r][d][(u,w)]  = (wd|ur)
//   OO[(q,r)][l'][z]  = (ql'|rz) for l' < no, -F_rz for l' = no
//   OV[(q,r)][0][(u,w)] = (qu|rw)
// and per triple in flight (slot) the contravariant amplitudes in three cyclic
// layouts V_L (slot L outermost = x, L+1 = y, L+2 = z innermost) with K blocks
// ordered (z block, y): read as rows x, K = (zb, y, zz) by the vvov and
// singles contractions, and as rows (y, x), K = z by the ooov and F ones.
// Zg, Zh and OV use the same (zb, u, zz) K order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dd.cuh"
#include "split.h"
#include "split_engine.h"
#include "split_kernels.h"

namespace cc3 {

#define CU(x)                                                              \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)
#define TRY(x)                  \
  do {                          \
    int r_ = (x);               \
    if (r_ != CC3_OK) return r_; \
  } while (0)

namespace {

// Slice-array descriptor: [slab][K/16][row group][slice][8 x 16 core-matrix pair]
SArr make_arr(const void *base, long long K, long long rps, long long slabs, int slices) {
  SArr a;
  a.base = reinterpret_cast<unsigned long long>(base);
  a.kblocks = (int)(K / 16);
  a.rows = (int)((rps + 7) / 8 * 8);
  a.slabs = (int)slabs;
  a.kb_stride = (long long)a.rows * 16 * slices;
  a.slab_stride = (long long)a.kblocks * a.kb_stride;
  return a;
}
size_t arr_elems(long long K, long long rps, long long slabs, int slices) {
  return (size_t)slices * slabs * (K / 16) * ((rps + 7) / 8 * 8) * 16;
}

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

int exponent_of(double mx) {
  if (!(mx > 0.0)) return 0;
  int e;
  std::frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  return e;
}

// N tile: at most S_NT_MAX (96) columns, a multiple of 16, balanced over tiles
int ntile_for(int N) {
  const int nt = (N + S_NT_MAX - 1) / S_NT_MAX;
  return std::min<int>(S_NT_MAX, rup((N + nt - 1) / nt, 16));
}

enum MapId {
  MA_T2S = 0, MA_T2C, MA_T2R, MA_XS, MA_YS, MA_OS, MA_V0, MA_V1, MA_V2, MA_V0K, MA_V1K, MA_V2K,
  MB_T2S, MB_T2C, MB_T2R, MB_XS, MB_YS, MB_OS, MB_ZG, MB_ZH, MB_OO, MB_OV,
  // Jacobian: per trial vector (R2 in the t2 layouts, g^ in the integral
  // layouts), F^ of all vectors, and ovov in the layouts of Algorithm 2
  MJ_R2S, MJ_R2C, MJ_R2R, MJ_XH, MJ_YH, MJ_OH, MJ_FH, MJ_OVD, MJ_OVZA, MJ_OVZB,
  // left transformation: t2 as [(p,q)][d][x] (G), as [p][l][(u,w)] in both K
  // orders (H), and Lt2 of every vector as [(p,q)][v][(u,w)] in both orders (Q)
  ML_T2T, ML_T2ZA, ML_T2ZB, ML_LQA, ML_LQB,
  // densities: t2 as [q][l][(u,w)] in both K orders (Y), and tau itself in the
  // rows-x views of the three cyclic layouts (D_vv)
  MD_T2YA, MD_T2YB, MD_TAU0, MD_TAU1, MD_TAU2,
  // the left transformation's Cholesky product: L^J_bd as [J][(b,d)] and one
  // vector's G as [(c,k)][(b,d)]
  ML_CHA, ML_GB,
  MAP_COUNT
};
static_assert((int)MAP_COUNT <= (int)SMAX_MAPS, "map table");

struct SplitState {
  int s = 0, vp = 0, op = 0, Et = 0, Eg = 0;
  int Nab = 0, N3 = 0, N1 = 16;
  __nv_bfloat16 *T2S = nullptr, *T2C = nullptr, *T2R = nullptr, *XS = nullptr, *YS = nullptr,
                *OS = nullptr, *Zg = nullptr, *Zh = nullptr, *OO = nullptr, *OV = nullptr;
  // Jacobian (Algorithm 2 layouts of ovov), staged on first use
  __nv_bfloat16 *OVD = nullptr, *OVZA = nullptr, *OVZB = nullptr;
  // Jacobian: the vv block of the Cholesky vectors, rows (b,d), K = J
  __nv_bfloat16 *LVV = nullptr;
  int EL = 0;
  int ks4 = 1;  // K split of the rows-x contractions
  // tunables (autotuner): K steps per vvov tile, N tile of the W build (0: default)
  int ks_target = 400, nt_w = 0;
  bool stack_vvov = true;  // stack permutations along M in the vvov contraction
  bool pair_ooov = true;   // one ooov job for the two permutations of a z slot
  // the residual's launch sequence as a CUDA graph (captured on the second
  // untraced call on a non-default stream, replayed afterwards)
  cudaGraphExec_t gexec = nullptr;
  long long g_launches = 0;
  int g_calls = 0;
  float2 *evdd = nullptr;
  int batch = 0;
  // per slot: the W build's partial sums (Wdd, TTdd, W3dd; tau~ replaces the
  // second), and e_i + e_j + e_k of every triple (dd) for the denominators
  float2 *Wdd = nullptr, *TTdd = nullptr, *W3dd = nullptr, *eo_tri = nullptr;
  __nv_bfloat16 *V[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16 **vptr = nullptr;  // device copy of {V[0..2]}
  unsigned int *maxbits = nullptr;
  int *slot_ex = nullptr;
  int *status = nullptr;
  SArrTable arrs;
  std::vector<SDevPlan> ab, om;
  std::vector<int> nslot;
  double executed = 0.0;
  bool staged = false, planned = false;
};

SplitState *state(cc3_ctx *c) { return reinterpret_cast<SplitState *>(c->split); }

template <class T>
int alloc(T **p, size_t n) {
  *p = nullptr;
  if (cudaMalloc(p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
    cudaGetLastError();
    return CC3_ERR_OOM;
  }
  return CC3_OK;
}

void drop_graph(SplitState *S) {
  if (S->gexec) cudaGraphExecDestroy(S->gexec);
  S->gexec = nullptr;
  S->g_calls = 0;
}

void free_state_buffers(SplitState *S) {
  drop_graph(S);
  void *bufs[] = {S->T2S, S->T2C, S->T2R, S->XS, S->YS, S->OS, S->Zg, S->Zh, S->OO, S->OV,
                  S->OVD, S->OVZA, S->OVZB, S->LVV, S->evdd, S->Wdd, S->TTdd, S->W3dd, S->eo_tri, S->V[0], S->V[1], S->V[2], S->vptr, S->maxbits,
                  S->slot_ex, S->status};
  for (void *p : bufs)
    if (p) cudaFree(p);
  for (auto *v : {&S->ab, &S->om})
    for (auto &d : *v) s_free_plan(&d);
}

// oo[(q,r)][l'][z] = ooov[q][l'][r][z] (l' < no), -F[r][z] (l' = no)
__global__ void build_oo_kernel(const double *__restrict__ ooov, const double *__restrict__ F,
                                double *__restrict__ oo, int no, int nv) {
  const long long n = (long long)no * no * (no + 1) * nv;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(e % nv);
    const int l = (int)((e / nv) % (no + 1));
    const long long qr = e / ((long long)nv * (no + 1));
    const int q = (int)(qr / no), r = (int)(qr % no);
    oo[e] = l < no ? ooov[(((long long)q * no + l) * no + r) * nv + z] : -F[(long long)r * nv + z];
  }
}

int stage(cc3_ctx *c, SplitState *S, cudaStream_t st) {
  const int no = c->no, nv = c->nv, s = S->s;
  S->vp = rup(nv, 16);
  S->op = rup(no, 16);
  const int vp = S->vp, op = S->op;
  const long long nv2 = (long long)nv * nv;
  // exponents of t2 and of all integral blocks (one common scale)
  unsigned long long *mx = nullptr;
  TRY(alloc(&mx, 8));
  CU(cudaMemsetAsync(mx, 0, 8 * sizeof(unsigned long long), st));
  TRY(launch_maxabs(c->t2, (long long)no * no * nv2, mx + 0, st));
  TRY(launch_maxabs(c->vvvo, nv2 * nv * no, mx + 1, st));
  TRY(launch_maxabs(c->ooov, (long long)no * no * no * nv, mx + 2, st));
  if (c->general) {  // the blocks the symmetric case derives from vvvo and ooov
    TRY(launch_maxabs(c->oovo, (long long)no * no * no * nv, mx + 2, st));
    TRY(launch_maxabs(c->vvov, nv2 * nv * no, mx + 1, st));
  }
  TRY(launch_maxabs(c->ovov, (long long)no * no * nv2, mx + 3, st));
  TRY(launch_maxabs(c->F_ov, (long long)no * nv, mx + 4, st));
  unsigned long long h[8];
  CU(cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  cudaFree(mx);
  double hv[5];
  for (int i = 0; i < 5; ++i) std::memcpy(&hv[i], &h[i], 8);
  S->Et = exponent_of(hv[0]);
  S->Eg = exponent_of(std::max(std::max(hv[1], hv[2]), std::max(hv[3], hv[4])));

  auto slab = [&](__nv_bfloat16 **dst, const double *src, long long rows, int Kp, int E,
                  const Gather &g, int rps) -> int {
    const size_t n = arr_elems(Kp, rps, rows / rps, s);
    TRY(alloc(dst, n));
    CU(cudaMemsetAsync(*dst, 0, n * sizeof(__nv_bfloat16), st));
    return launch_slice_gather(src, *dst, s, E, g, rows, Kp, rps, st);
  };
  Gather g;
  // T2S[(p,q)][x][d] = t2[p][q][x][d]
  g = {0, (long long)no * nv2, nv2, nv, 0, 1, no, nv, vp, nv, 1};
  TRY(slab(&S->T2S, c->t2, (long long)no * no * nv, vp, S->Et, g, nv));
  // T2C[(p,y)][x][l] = t2[p][l][x][y]
  g = {0, (long long)no * nv2, 1, nv, 0, nv2, nv, nv, op, no, 1};
  TRY(slab(&S->T2C, c->t2, (long long)no * nv * nv, op, S->Et, g, nv));
  // T2R[(p,x)][y][l] = t2[p][l][x][y]
  g = {0, (long long)no * nv2, nv, 1, 0, nv2, nv, nv, op, no, 1};
  TRY(slab(&S->T2R, c->t2, (long long)no * nv * nv, op, S->Et, g, nv));
  // XS[(r,z)][y][d] = vvvo[y][d][z][r]
  g = {0, 1, no, nv2 * no, 0, (long long)nv * no, nv, nv, vp, nv, 1};
  TRY(slab(&S->XS, c->vvvo, (long long)no * nv * nv, vp, S->Eg, g, nv));
  // YS[(r,y)][z][d] = vvvo[y][d][z][r]
  g = {0, 1, nv2 * no, no, 0, (long long)nv * no, nv, nv, vp, nv, 1};
  TRY(slab(&S->YS, c->vvvo, (long long)no * nv * nv, vp, S->Eg, g, nv));
  // OS[(q,r)][z][l] = oovo[l][q][z][r]
  g = {0, (long long)nv * no, 1, no, 0, (long long)no * nv * no, no, nv, op, no, 1};
  TRY(slab(&S->OS, c->oovo, (long long)no * no * nv, op, S->Eg, g, nv));
  // Zg[r][d][(u,w)] = g_durw, Zh[r][d][(u,w)] = g_dwru: from vvov[d][b][k][c]
  // for general integrals, else through the symmetry g_durw = vvvo[u][d][w][r]
  // (Zg) and g_dwru = vvvo[w][d][u][r] (Zh)
  if (c->general) {
    const long long sd = (long long)nv * no * nv, sb = (long long)no * nv;
    g = {0, 0, nv, sd, sb, 1, no, nv, nv, nv, nv, 1};
    TRY(slab(&S->Zg, c->vvov, (long long)no * nv, nv * vp, S->Eg, g, nv));
    g = {0, 0, nv, sd, 1, sb, no, nv, nv, nv, nv, 1};
    TRY(slab(&S->Zh, c->vvov, (long long)no * nv, nv * vp, S->Eg, g, nv));
  } else {
    g = {0, 0, 1, (long long)nv * no, nv2 * no, no, no, nv, nv, nv, nv, 1};
    TRY(slab(&S->Zg, c->vvvo, (long long)no * nv, nv * vp, S->Eg, g, nv));
    g = {0, 0, 1, (long long)nv * no, no, nv2 * no, no, nv, nv, nv, nv, 1};
    TRY(slab(&S->Zh, c->vvvo, (long long)no * nv, nv * vp, S->Eg, g, nv));
  }
  // OO[(q,r)][l'][z]
  {
    double *oo = nullptr;
    const long long n = (long long)no * no * (no + 1) * nv;
    TRY(alloc(&oo, n));
    build_oo_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(
        c->ooov, c->F_ov, oo, no, nv);
    CU(cudaGetLastError());
    // rows ((q,r), l') flattened and contiguous: r0 = row, stride nv
    g = {0, 0, 0, nv, 0, 1, 1, 1 << 30, vp, nv, 1};
    TRY(slab(&S->OO, oo, (long long)no * no * (no + 1), vp, S->Eg, g, no + 1));
    CU(cudaStreamSynchronize(st));
    cudaFree(oo);
  }
  // OV[(q,r)][0][(u,w)] = ovov[q][u][r][w]
  g = {0, 0, (long long)nv * no * nv, nv, (long long)no * nv, 1, no, no, nv, nv, nv, 1};
  TRY(slab(&S->OV, c->ovov, (long long)no * no, nv * vp, S->Eg, g, 1));
  // dd orbital energies
  {
    std::vector<double> ev(nv);
    CU(cudaMemcpyAsync(ev.data(), c->eps_v, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    std::vector<float2> evd(nv);
    for (int a = 0; a < nv; ++a) {
      dd::df x = dd::from_double_host(ev[a]);
      evd[a] = make_float2(x.hi, x.lo);
    }
    TRY(alloc(&S->evdd, (size_t)nv));
    CU(cudaMemcpyAsync(S->evdd, evd.data(), sizeof(float2) * nv, cudaMemcpyHostToDevice, st));
  }
  // per-batch workspace
  const double per_slot = (double)nv2 * nv * 24.0 + 3.0 * s * nv2 * vp * 2.0;
  S->batch = (int)std::max(1.0, std::min(16.0, 6.0e9 / per_slot));
  S->batch = std::min(S->batch, std::max(1, c->ntri));
  const size_t nb = (size_t)S->batch;
  TRY(alloc(&S->Wdd, nb * nv2 * nv));
  TRY(alloc(&S->TTdd, nb * nv2 * nv));
  TRY(alloc(&S->W3dd, nb * nv2 * nv));
  for (int L = 0; L < 3; ++L) {
    const size_t n4 = arr_elems((long long)nv * vp, nv, (long long)nb, s);
    TRY(alloc(&S->V[L], n4));
    CU(cudaMemsetAsync(S->V[L], 0, n4 * sizeof(__nv_bfloat16), st));
  }
  {
    __nv_bfloat16 *h[3] = {S->V[0], S->V[1], S->V[2]};
    TRY(alloc(&S->vptr, 3));
    CU(cudaMemcpyAsync(S->vptr, h, sizeof(h), cudaMemcpyHostToDevice, st));
  }
  TRY(alloc(&S->maxbits, nb));
  TRY(alloc(&S->slot_ex, nb));
  TRY(alloc(&S->status, 4));
  CU(cudaMemsetAsync(S->status, 0, 4 * sizeof(int), st));

  // slice-array table (the same descriptor serves an array as A or B operand)
  S->Nab = S->nt_w > 0 ? S->nt_w : ntile_for(nv);
  S->N3 = rup(no + 1, 16);
  if (S->N3 > S_NT_MAX) return CC3_ERR_UNSUPPORTED;
  SArr *M = S->arrs.a;
  std::memset(&S->arrs, 0, sizeof(S->arrs));
  const long long n_o = no, n_v = nv;
  M[MA_T2S] = M[MB_T2S] = make_arr(S->T2S, vp, n_v, n_o * n_o, s);
  M[MA_T2C] = M[MB_T2C] = make_arr(S->T2C, op, n_v, n_o * n_v, s);
  M[MA_T2R] = M[MB_T2R] = make_arr(S->T2R, op, n_v, n_o * n_v, s);
  M[MA_XS] = M[MB_XS] = make_arr(S->XS, vp, n_v, n_o * n_v, s);
  M[MA_YS] = M[MB_YS] = make_arr(S->YS, vp, n_v, n_o * n_v, s);
  M[MA_OS] = M[MB_OS] = make_arr(S->OS, op, n_v, n_o * n_o, s);
  const long long nv8 = (n_v + 7) / 8 * 8;
  for (int L = 0; L < 3; ++L) {
    M[MA_V0 + L] = make_arr(S->V[L], n_v * vp, n_v, (long long)nb, s);        // rows x, K = (zb, y, zz)
    M[MA_V0K + L] = make_arr(S->V[L], vp, n_v * nv8, (long long)nb, s);       // rows (y, x), K = z
  }
  M[MB_ZG] = make_arr(S->Zg, n_v * vp, n_v, n_o, s);
  M[MB_ZH] = make_arr(S->Zh, n_v * vp, n_v, n_o, s);
  M[MB_OO] = make_arr(S->OO, vp, n_o + 1, n_o * n_o, s);
  M[MB_OV] = make_arr(S->OV, n_v * vp, 1, n_o * n_o, s);
  CU(cudaStreamSynchronize(st));
  S->staged = true;
  return CC3_OK;
}

// ---- plans --------------------------------------------------------------------
SOpnd opd(int map, int slab0, int slab_b = 0, int row0 = 0, int row_b = 0) {
  SOpnd o;
  o.map = map;
  o.slab0 = slab0;
  o.slab_b = slab_b;
  o.row0 = row0;
  o.row_b = row_b;
  return o;
}
OutD outd(int buf, long long off, long long sm0, long long sn0, long long sb = 0) {
  OutD c;
  c.buf = buf;
  c.m_in = 1 << 30;
  c.n_in = 1 << 30;
  c.off = off;
  c.sb = sb;
  c.sm1 = 0;
  c.sm0 = sm0;
  c.sn1 = 0;
  c.sn0 = sn0;
  return c;
}

int new_sjob(SPlan &P, int M, int N, int Ntile, int batch, int ksplit, int mode, int expo,
             double &executed, int slices) {
  SJob j;
  std::memset(&j, 0, sizeof(j));
  j.M = M;
  j.N = N;
  j.Nm = N;
  j.n_valid = N;
  j.Ntile = Ntile;
  j.batch = batch;
  j.ksplit = std::max(1, ksplit);
  j.mode = mode;
  j.expo = expo;
  j.expo_slot = -1;
  j.expo_slot2 = -1;
  j.mult = 1.0f;
  j.tiles_m = (M + S_BM - 1) / S_BM;
  j.tiles_n = (N + Ntile - 1) / Ntile;
  j.term0 = (int)P.terms.size();
  j.nterm = 0;
  j.tile_base = P.tiles;
  P.tiles += (long long)batch * j.tiles_m * j.tiles_n * j.ksplit;
  P.jobs.push_back(j);
  (void)executed;
  (void)slices;
  return (int)P.jobs.size() - 1;
}
void add_sterm(SPlan &P, int job, SOpnd A, SOpnd B, int K, int negA, double &executed,
               int slices, const SOpnd *Bt = nullptr, int nbm = 0) {
  STerm t;
  std::memset(&t, 0, sizeof(t));
  t.A = A;
  t.B = B;
  t.Bt = Bt ? *Bt : B;
  t.nbm = Bt ? nbm : 0;
  t.ksteps = K / S_BK;
  t.negA = negA;
  P.terms.push_back(t);
  SJob &j = P.jobs[job];
  j.nterm++;
  executed += 2.0 * j.tiles_m * S_BM * (double)j.tiles_n * j.Ntile * K * j.batch *
              (slices * (slices + 1) / 2);
  const double mrows = j.m_pad > 0 ? (double)(j.M / j.m_pad) * j.m_valid +
                                        std::min(j.M % j.m_pad, j.m_valid)
                                  : (double)j.M;
  const double ncols = j.route == 1 ? 2.0 * (j.Nm + j.tw) : (double)(j.n_valid + (j.N - j.Nm));
  const double useful = 2.0 * mrows * ncols * K * j.batch;
  P.flop += useful;
  P.slice_flop += useful * (slices * (slices + 1) / 2);
}

// Slice arrays that play t2 and the (vvvo, oovo) integrals in the W build
// (the same descriptor serves as A or B operand).
// The slab offsets select one trial vector's part of an array that holds the
// slices of every vector back to back (the Jacobian's R2 and g^ arrays): t2
// roles (S, C, R layouts) and integral roles (XS, YS, OS layouts).
struct WMaps {
  int aT2S, bT2S, aT2C, bT2C, aT2R, bT2R, aXS, bXS, aYS, bYS, aOS, bOS;
  int oS = 0, oC = 0, oR = 0, oXS = 0, oYS = 0, oOS = 0;
};
const WMaps kStdMaps = {MA_T2S, MB_T2S, MA_T2C, MB_T2C, MA_T2R, MB_T2R,
                        MA_XS,  MB_XS,  MA_YS,  MB_YS,  MA_OS,  MB_OS};

// W build of triple (i,j,k) in three phases.  Every term has one operand
// that carries a virtual index besides the tile's two (t2 / integral slabs
// (x, 0..nv-1)); it is the A operand, its nv slabs read as one array of
// nv * rows flattened rows (rows: the slab's row count, nv padded to 8), so
// the tiles cover the nv^2 x nv block of W without M padding.
//   phase 1: rows (c, a), columns b -> W_1[c][a][b]
//   phase 2: rows (c, b), columns a -> W_2[c][a][b]
//   phase 3: rows (a, b), columns c -> W_3[c][a][b]
// The three phases write separate buffers (W_2 in the tau~ workspace), so one
// launch runs them all; the element-wise step forms tau = (W_1 + W_2 + W_3) /
// (w - eps) and tau~ from the three.
int w_job(SPlan &P, int nv, int rows, int Nt, int phase, int slot, int E, double &ex, int s) {
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const int jb = new_sjob(P, nv * rows, nv, Nt, 1, 1, SEPI_DD_STORE, E, ex, s);
  SJob &J = P.jobs[jb];
  OutD C = outd(phase == 1 ? B_WS_W : (phase == 2 ? B_WS_TT : B_WS_W3), slot * nv3, 0, 0);
  C.m_in = rows;
  if (phase == 1) {
    C.sm1 = nv2, C.sm0 = nv, C.sn0 = 1;
  } else if (phase == 2) {
    C.sm1 = nv2, C.sm0 = 1, C.sn0 = nv;
  } else {
    C.sm1 = nv, C.sm0 = 1, C.sn0 = nv2;
  }
  J.C = C;
  J.Ct = C;
  J.m_pad = rows;
  J.m_valid = nv;
  J.nv = nv;
  return jb;
}
// A: slabs (x, 0..nv-1) of map `am` flattened; B: slab `bslab` of map `bm`
void w_term(SPlan &P, int jb, int am, int x, int bm, int bslab, int K, int neg, int nv,
            int rows, double &ex, int s, int aoff = 0, int boff = 0) {
  add_sterm(P, jb, opd(am, aoff + x * nv), opd(bm, boff + bslab), K, neg, ex, s);
  P.terms.back().aflat = nv * rows;
}
// phase 1, rows (c, a), columns b:
//   sum_d (ad|ck) t^{bd}_{ji} [X_k],  sum_d (cd|ai) t^{bd}_{jk} [Y_i],
//   -sum_l t^{ca}_{kl} (li|bj) [T2R_k],  -sum_l t^{ac}_{il} (lk|bj) [T2C_i]
void w_terms_1(SPlan &P, int jb, const WMaps &m, int no, int nv, int rows, int vp, int op,
               const int ijk[3], double &ex, int s) {
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  w_term(P, jb, m.aXS, k, m.bT2S, j * no + i, vp, 0, nv, rows, ex, s, m.oXS, m.oS);
  w_term(P, jb, m.aYS, i, m.bT2S, j * no + k, vp, 0, nv, rows, ex, s, m.oYS, m.oS);
  w_term(P, jb, m.aT2R, k, m.bOS, i * no + j, op, 1, nv, rows, ex, s, m.oR, m.oOS);
  w_term(P, jb, m.aT2C, i, m.bOS, k * no + j, op, 1, nv, rows, ex, s, m.oC, m.oOS);
}
// phase 2, rows (c, b), columns a: the terms whose t2 / oovo factor carries a
void w_terms_2(SPlan &P, int jb, const WMaps &m, int no, int nv, int rows, int vp, int op,
               const int ijk[3], double &ex, int s) {
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  w_term(P, jb, m.aXS, k, m.bT2S, i * no + j, vp, 0, nv, rows, ex, s, m.oXS, m.oS);
  w_term(P, jb, m.aYS, j, m.bT2S, i * no + k, vp, 0, nv, rows, ex, s, m.oYS, m.oS);
  w_term(P, jb, m.aT2C, j, m.bOS, k * no + i, op, 1, nv, rows, ex, s, m.oC, m.oOS);
  w_term(P, jb, m.aT2R, k, m.bOS, j * no + i, op, 1, nv, rows, ex, s, m.oR, m.oOS);
}
// phase 3, rows (a, b), columns c: the terms whose t2 / oovo factor carries c
void w_terms_3(SPlan &P, int jc, const WMaps &m, int no, int nv, int rows, int vp, int op,
               const int ijk[3], double &ex, int s) {
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  // (k,i,j): sum_d t_ki[c][d] (ad|bj) -> YS slabs (j, a) rows b
  w_term(P, jc, m.aYS, j, m.bT2S, k * no + i, vp, 0, nv, rows, ex, s, m.oYS, m.oS);
  // (k,j,i): sum_d t_kj[c][d] (bd|ai) -> XS slabs (i, a) rows b
  w_term(P, jc, m.aXS, i, m.bT2S, k * no + j, vp, 0, nv, rows, ex, s, m.oXS, m.oS);
  // (i,j,k) occupied: - sum_l (lj|ck) t^{ab}_{il} -> T2R slabs (i, a) rows b
  w_term(P, jc, m.aT2R, i, m.bOS, j * no + k, op, 1, nv, rows, ex, s, m.oR, m.oOS);
  // (j,i,k) occupied: - sum_l (li|ck) t^{ba}_{jl} -> T2C slabs (j, a) rows b
  w_term(P, jc, m.aT2C, j, m.bOS, i * no + k, op, 1, nv, rows, ex, s, m.oC, m.oOS);
}

// the three W build phases of one triple (one launch)
void plan_w_split(SPlan &pab, SplitState *S, int no, int nv, const int ijk[3], int slot,
                  double &ex) {
  const int s = S->s, E = S->Et + S->Eg - 14, rows = (nv + 7) / 8 * 8;
  const int j1 = w_job(pab, nv, rows, S->Nab, 1, slot, E, ex, s);
  w_terms_1(pab, j1, kStdMaps, no, nv, rows, S->vp, S->op, ijk, ex, s);
  const int j2 = w_job(pab, nv, rows, S->Nab, 2, slot, E, ex, s);
  w_terms_2(pab, j2, kStdMaps, no, nv, rows, S->vp, S->op, ijk, ex, s);
  const int j3 = w_job(pab, nv, rows, S->Nab, 3, slot, E, ex, s);
  w_terms_3(pab, j3, kStdMaps, no, nv, rows, S->vp, S->op, ijk, ex, s);
}

// Appends the jobs of src to dst (one launch runs dst's jobs in order).
void append_plan(SPlan &dst, const SPlan &src) {
  const int t0 = (int)dst.terms.size();
  for (SJob j : src.jobs) {
    j.term0 += t0;
    j.tile_base += dst.tiles;
    dst.jobs.push_back(j);
  }
  dst.terms.insert(dst.terms.end(), src.terms.begin(), src.terms.end());
  dst.tiles += src.tiles;
  dst.flop += src.flop;
  dst.slice_flop += src.slice_flop;
}

// residual contractions of one triple (every distinct permutation); which:
// bit 0 the vvov + singles jobs (long K), bit 1 the ooov + F jobs (short K),
// bit 3 leave out the singles and F columns (the left transformation's sigma2
// contractions)
void plan_omega_split(SPlan &P, SplitState *S, int no, int nv, const int ijk[3], int slot,
                      int ksplit4, double &ex, int which = 3) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const int s = S->s, vp = S->vp;
  const long long nv2 = (long long)nv * nv;
  const int E = S->Eg - 14;  // + slot exponent of tau~
  int seen[6][3], nseen = 0;
  int ooov[6][5], nooov = 0;  // (p, q, r, Lz, xouter) of the ooov / F jobs
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int u = 0; u < 6; ++u) {
    const int *m = PERM6[u];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int w = 0; w < nseen; ++w)
      if (seen[w][0] == p && seen[w][1] == q && seen[w][2] == r) dup = true;
    if (dup) continue;
    seen[nseen][0] = p;
    seen[nseen][1] = q;
    seen[nseen][2] = r;
    ++nseen;
    // layout with x slot outermost: K order (slot m0+1, slot m0+2)
    const int L = m[0];
    const bool yz = (m[1] == (L + 1) % 3);
    if ((which & 1) && (which & 8)) {  // the vvov contraction alone
      int jb = new_sjob(P, nv, nv, ntile_for(nv), 1, ksplit4, SEPI_F64_ATOMIC, E, ex, s);
      P.jobs[jb].expo_slot = slot;
      P.jobs[jb].C = outd(B_OMT, ((long long)p * no + q) * nv2, nv, 1);
      P.jobs[jb].Ct = P.jobs[jb].C;
      add_sterm(P, jb, opd(MA_V0 + L, slot), opd(yz ? MB_ZG : MB_ZH, r), nv * vp, 0, ex, s);
    } else if (which & 1) {  // Omega~^{ad}_{pq} += sum_{yz} V[x][y][z] (dy|rz)   columns d < nv
       // Omega1^x_p       += sum_{yz} V[x][y][z] (qy|rz)   tail column nv8
      const int nv8 = (nv + 7) / 8 * 8;
      int jb = new_sjob(P, nv, nv8 + 1, ntile_for(nv8 + 1), 1, ksplit4, SEPI_F64_ATOMIC, E, ex, s);
      P.jobs[jb].expo_slot = slot;
      P.jobs[jb].Nm = nv8;
      P.jobs[jb].n_valid = nv;
      P.jobs[jb].C = outd(B_OMT, ((long long)p * no + q) * nv2, nv, 1);
      P.jobs[jb].Ct = outd(B_OM1, (long long)p * nv, 1, 0);
      const SOpnd tail = opd(MB_OV, yz ? q * no + r : r * no + q);
      add_sterm(P, jb, opd(MA_V0 + L, slot), opd(yz ? MB_ZG : MB_ZH, r), nv * vp, 0, ex, s,
                &tail, nv8);
    }
    if (which & 2) {  // the ooov / F job, formed below
      ooov[nooov][0] = p;
      ooov[nooov][1] = q;
      ooov[nooov][2] = r;
      ooov[nooov][3] = (m[2] + 1) % 3;  // Lz
      ooov[nooov][4] = m[0] == (m[2] + 1) % 3 ? 1 : 0;  // xouter
      ++nooov;
    }
  }
  // Omega~^{xy}_{pl} -= sum_z V (ql|rz);  Omega~^{xy}_{pq} += sum_z V F_rz.
  // Layout Lz has z innermost; its rows (y_L, x_L) are the perm's (y, x) when
  // the perm's x slot is Lz (xouter), else (x, y); row m = y_L * nv8 + x_L.
  // The two permutations with the same z slot read the same tau~ rows (layout
  // Lz): when the columns allow, one job takes both, B rows [0, cs) from the
  // first permutation's OO block and [cs, 2 cs) from the second's.
  const int nv8 = (nv + 7) / 8 * 8, cs = (no + 1 + 7) / 8 * 8;
  const bool pair_ok = S->pair_ooov && (cs + no + 1 + 15) / 16 * 16 <= S_NT_MAX;
  auto ooov_out = [&](int p, int xo, int l0, OutD *c, OutD *ct) {
    // Omega~[p][l][x][y] at x*nv + y; the tail column is l = l0
    *c = outd(B_OMT, (long long)p * no * nv2, xo ? nv : 1, nv2);
    c->m_in = nv8;
    c->sm1 = xo ? 1 : nv;
    *ct = outd(B_OMT, ((long long)p * no + l0) * nv2, xo ? nv : 1, 0);
    ct->m_in = nv8;
    ct->sm1 = xo ? 1 : nv;
  };
  bool used[6] = {false, false, false, false, false, false};
  for (int a = 0; a < nooov; ++a) {
    if (used[a]) continue;
    used[a] = true;
    int b = -1;
    for (int u = a + 1; u < nooov && pair_ok; ++u)
      if (!used[u] && ooov[u][3] == ooov[a][3]) {
        b = u;
        break;
      }
    const int Lz = ooov[a][3];
    const bool notail = (which & 8) != 0;
    if (b < 0) {
      // without the F column the job stops at the last ooov row of OO
      int jb = new_sjob(P, nv * nv8, notail ? no : no + 1, S->N3, 1, 1, SEPI_F64_ATOMIC, E, ex,
                        s);
      SJob &J = P.jobs[jb];
      J.expo_slot = slot;
      J.Nm = no;
      J.m_pad = nv8;
      J.m_valid = nv;
      ooov_out(ooov[a][0], ooov[a][4], ooov[a][1], &J.C, &J.Ct);
      add_sterm(P, jb, opd(MA_V0K + Lz, slot), opd(MB_OO, ooov[a][1] * no + ooov[a][2]), vp, 1,
                ex, s);
      continue;
    }
    used[b] = true;
    const int N = cs + no + 1;
    int jb = new_sjob(P, nv * nv8, N, (N + 15) / 16 * 16, 1, 1, SEPI_F64_ATOMIC, E, ex, s);
    SJob &J = P.jobs[jb];
    J.expo_slot = slot;
    J.Nm = no;
    J.n_valid = N;
    J.route = 1;  // columns [0, cs): first permutation, [cs, N): second
    J.Nm2 = cs;
    J.tw = notail ? 0 : 1;  // tw = 0: the F columns are computed and dropped
    J.m_pad = nv8;
    J.m_valid = nv;
    ooov_out(ooov[a][0], ooov[a][4], ooov[a][1], &J.C, &J.Ct);
    ooov_out(ooov[b][0], ooov[b][4], ooov[b][1], &J.C2, &J.Ct2);
    const SOpnd tail = opd(MB_OO, ooov[b][1] * no + ooov[b][2]);
    add_sterm(P, jb, opd(MA_V0K + Lz, slot), opd(MB_OO, ooov[a][1] * no + ooov[a][2]), vp, 1,
              ex, s, &tail, cs);
  }
}

// One distinct permutation of a triple in flight, as the vvov contraction
// sees it: the tau~ layout L whose rows are x, the K order flag and the
// output / integral indices.
struct VvovPerm {
  int slot, L, yz, p, q, r;
  long long omt_off = 0, om1_off = 0;  // output base of this permutation's vector
};

void collect_vvov_perms(std::vector<VvovPerm> &out, const int ijk[3], int slot) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  int seen[6][3], nseen = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int u = 0; u < 6; ++u) {
    const int *m = PERM6[u];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int w = 0; w < nseen; ++w)
      if (seen[w][0] == p && seen[w][1] == q && seen[w][2] == r) dup = true;
    if (dup) continue;
    seen[nseen][0] = p;
    seen[nseen][1] = q;
    seen[nseen][2] = r;
    ++nseen;
    const int L = m[0];
    VvovPerm v;
    v.slot = slot;
    v.L = L;
    v.yz = m[1] == (L + 1) % 3 ? 1 : 0;
    v.p = p;
    v.q = q;
    v.r = r;
    out.push_back(v);
  }
}

// The vvov + singles contraction of a batch with the permutations that share
// the integral operand (same r and K order) stacked along M: their x rows
// (nv each) are laid end to end and cut into 128-row tiles, so a tile may hold
// the last rows of one permutation and the first rows of the next (two A
// segments, two output row ranges, one singles tail column each).  Without
// stacking nv = 160 costs two 128-row tiles per permutation, 96 rows of
// padding in the second; with it, 1.25.  Needs nv a multiple of 8 and >= 128
// (a tile then spans at most two permutations).
void plan_vvov_stacked(SPlan &P, SplitState *S, int no, int nv, std::vector<VvovPerm> perms,
                       int ksplit4, double &ex) {
  const int s = S->s, vp = S->vp;
  const long long nv2 = (long long)nv * nv;
  std::stable_sort(perms.begin(), perms.end(), [](const VvovPerm &a, const VvovPerm &b) {
    return a.r != b.r ? a.r < b.r : a.yz < b.yz;
  });
  size_t g0 = 0;
  while (g0 < perms.size()) {
    size_t g1 = g0;
    while (g1 < perms.size() && perms[g1].r == perms[g0].r && perms[g1].yz == perms[g0].yz) ++g1;
    const long long total = (long long)(g1 - g0) * nv;
    for (long long R = 0; R < total; R += S_BM) {
      const size_t k = g0 + (size_t)(R / nv);
      const int x0 = (int)(R % nv);
      const int rows0 = (int)std::min<long long>(std::min<long long>(nv - x0, S_BM), total - R);
      const int rows1 = (rows0 < S_BM && k + 1 < g1) ? std::min(S_BM - rows0, nv) : 0;
      const VvovPerm &u = perms[k];
      const int N = rows1 > 0 ? nv + 9 : nv + 1;
      int jb = new_sjob(P, rows0 + rows1, N, ntile_for(N), 1, ksplit4, SEPI_F64_ATOMIC,
                        S->Eg - 14, ex, s);
      SJob &J = P.jobs[jb];
      J.expo_slot = u.slot;
      J.Nm = nv;
      J.n_valid = nv;
      J.C = outd(B_OMT, u.omt_off + (((long long)u.p * no + u.q) * nv + x0) * nv, nv, 1);
      J.Ct = outd(B_OM1, u.om1_off + (long long)u.p * nv + x0, 1, 0);
      const SOpnd tail = opd(MB_OV, u.yz ? u.q * no + u.r : u.r * no + u.q);
      add_sterm(P, jb, opd(MA_V0 + u.L, u.slot, 0, x0, 0), opd(u.yz ? MB_ZG : MB_ZH, u.r), nv * vp,
                0, ex, s, &tail, nv);
      if (rows1 > 0) {
        const VvovPerm &w = perms[k + 1];
        J.msplit = rows0;
        J.Nm2 = nv + 8;
        J.expo_slot2 = w.slot;
        J.C2 = outd(B_OMT, w.omt_off + ((long long)w.p * no + w.q) * nv2, nv, 1);
        J.Ct2 = outd(B_OM1, w.om1_off + (long long)w.p * nv, 1, 0);
        STerm &T = P.terms.back();
        T.A2 = opd(MA_V0 + w.L, w.slot);
        T.asplit = rows0;
        T.Bt2 = opd(MB_OV, w.yz ? w.q * no + w.r : w.r * no + w.q);
        T.nbm2 = nv + 8;
      }
    }
    g0 = g1;
  }
}

int build_plans(cc3_ctx *c, SplitState *S, cudaStream_t st) {
  drop_graph(S);
  for (auto *v : {&S->ab, &S->om})
    for (auto &d : *v) s_free_plan(&d);
  S->ab.clear();
  S->om.clear();
  S->nslot.clear();
  const int no = c->no, nv = c->nv;
  std::vector<double> eo(no);
  CU(cudaMemcpyAsync(eo.data(), c->eps_o, sizeof(double) * no, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  {  // e_i + e_j + e_k of every triple (dd), read by the element-wise step
    std::vector<float2> eot(std::max(1, c->ntri));
    for (int t = 0; t < c->ntri; ++t) {
      const int *ijk = &c->tri_host[3 * t];
      const dd::df ed = dd::from_double_host(eo[ijk[0]] + eo[ijk[1]] + eo[ijk[2]]);
      eot[t] = make_float2(ed.hi, ed.lo);
    }
    if (S->eo_tri) cudaFree(S->eo_tri);
    S->eo_tri = nullptr;
    TRY(alloc(&S->eo_tri, eot.size()));
    CU(cudaMemcpyAsync(S->eo_tri, eot.data(), sizeof(float2) * eot.size(),
                       cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
  }
  double ex = 0.0;
  // K split of the vvov contraction: tiles of about 400 K steps, so that the
  // persistent engine balances them over the SMs (partial sums add in FP64)
  const int kst = nv * S->vp / S_BK;
  int ks4 = std::max(1, (kst + S->ks_target - 1) / std::max(16, S->ks_target));
  S->ks4 = ks4;
  S->Nab = S->nt_w > 0 ? S->nt_w : ntile_for(nv);
  // stacked vvov tiles (see plan_vvov_stacked) where they save padding rows
  const bool stack = S->stack_vvov && nv >= S_BM && nv % 8 == 0 && nv % S_BM != 0;
  for (int t0 = 0; t0 < c->ntri; t0 += S->batch) {
    const int t1 = std::min(c->ntri, t0 + S->batch);
    SPlan pab, pom, pom3;
    std::vector<VvovPerm> vperms;
    for (int t = t0; t < t1; ++t) {
      const int *ijk = &c->tri_host[3 * t];
      plan_w_split(pab, S, no, nv, ijk, t - t0, ex);
      // the long-K tiles first: the persistent engine hands tiles out in order
      if (stack) {
        collect_vvov_perms(vperms, ijk, t - t0);
      } else {
        plan_omega_split(pom, S, no, nv, ijk, t - t0, ks4, ex, 1);
      }
      plan_omega_split(pom3, S, no, nv, ijk, t - t0, ks4, ex, 2);
    }
    if (stack) plan_vvov_stacked(pom, S, no, nv, vperms, ks4, ex);
    append_plan(pom, pom3);
    S->ab.emplace_back();
    S->om.emplace_back();
    TRY(s_upload_plan(pab, &S->ab.back(), st));
    TRY(s_upload_plan(pom, &S->om.back(), st));
    S->nslot.push_back(t1 - t0);
  }
  S->executed = ex;
  S->planned = true;
  return CC3_OK;
}

void fill_vptrs(cc3_ctx *c, SplitState *S, VPtrTable *P) {
  std::memset(P, 0, sizeof(*P));
  P->p[B_WS_W] = S->Wdd;
  P->p[B_WS_TT] = S->TTdd;  // W_2 of the W build until tau~ overwrites it
  P->p[B_WS_W3] = S->W3dd;
  P->p[B_EPSV] = S->evdd;
  P->p[B_OMT] = c->omt;
  P->p[B_OM1] = c->om1;
  P->fx[B_OMT] = c->omt_fx;  // null unless CC3_DETERMINISTIC
  P->fx[B_OM1] = c->om1_fx;
  P->p[B_SLOTEXP] = S->slot_ex;
}

}  // namespace

namespace {
// Tuned parameters per (no, nv, slices), shared by all contexts of the process.
struct TuneKey {
  int no, nv, s;
  bool operator<(const TuneKey &o) const {
    return no != o.no ? no < o.no : (nv != o.nv ? nv < o.nv : s < o.s);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tuned;  // -> (ks_target, nt_w)

// The staged slice arrays and residual plans of the context (built on first use).
int split_ready(cc3_ctx *c, SplitState **out, cudaStream_t st) {
  const int s = c->slices > 0 ? c->slices : 6;
  SplitState *S = state(c);
  if (S && S->s != s) {
    split_destroy(c);
    S = nullptr;
  }
  if (!S) {
    S = new (std::nothrow) SplitState();
    if (!S) return CC3_ERR_OOM;
    S->s = s;
    c->split = S;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey{c->no, c->nv, s});
    if (it != g_tuned.end()) {
      S->ks_target = it->second.first;
      S->nt_w = it->second.second;
    }
  }
  if (!S->staged) TRY(stage(c, S, st));
  if (!S->planned) TRY(build_plans(c, S, st));
  *out = S;
  return CC3_OK;
}
}  // namespace

namespace {
// The residual's launch sequence: per batch of triples the W build (one
// launch, three partial sums), tau and tau~ from them, the slices of tau~,
// and the contractions.
int omega_sequence(cc3_ctx *c, SplitState *S, cudaStream_t st) {
  const int s = S->s;
  VPtrTable P;
  fill_vptrs(c, S, &P);
  const int nv = c->nv;
  const int kdrain = S_DRAIN_STEPS;
  for (size_t b = 0, t0 = 0; b < S->ab.size(); t0 += S->nslot[b], ++b) {
    const int ns = S->nslot[b];
    trace_begin(c, TR_SPLIT_W, st);
    TRY(s_launch_plan(S->ab[b], S->arrs, P, s, kdrain, S->status, st, &c->counters.launches));
    trace_end(c, TR_SPLIT_W, st, S->ab[b].flop, S->ab[b].slice_flop);
    trace_begin(c, TR_SPLIT_ELEM, st);
    CU(cudaMemsetAsync(S->maxbits, 0, sizeof(unsigned int) * ns, st));
    TRY(launch_tau_contravariant_dd(S->Wdd, S->TTdd, S->W3dd, S->TTdd, S->evdd, S->eo_tri + t0,
                                    0.f, 0.f, nv, ns, S->maxbits, st));
    TRY(launch_slot_exponent(S->maxbits, S->slot_ex, ns, st));
    TRY(launch_slice_tt(S->TTdd, S->vptr, nv, S->vp, s, S->slot_ex, ns, S->batch, st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    c->counters.launches += 3;
    trace_begin(c, TR_SPLIT_OMEGA, st);
    TRY(s_launch_plan(S->om[b], S->arrs, P, s, kdrain, S->status, st, &c->counters.launches));
    trace_end(c, TR_SPLIT_OMEGA, st, S->om[b].flop, S->om[b].slice_flop);
  }
  return CC3_OK;
}
}  // namespace

int split_omega(cc3_ctx *c, cudaStream_t st) {
  SplitState *S = nullptr;
  TRY(split_ready(c, &S, st));
  const int s = S->s;
  // untraced calls on a stream other than the legacy default one replay a
  // captured graph of the whole sequence (the plans and buffers it uses are
  // fixed until the plans are rebuilt)
  const bool graphable = !c->trace.on && st != nullptr && st != cudaStreamLegacy;
  if (graphable && S->gexec) {
    CU(cudaGraphLaunch(S->gexec, st));
    c->counters.launches += S->g_launches;
  } else if (graphable && S->g_calls >= 1) {
    const long long before = c->counters.launches;
    CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = omega_sequence(c, S, st);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc == CC3_OK && ec == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
      S->gexec = exec;
      S->g_launches = c->counters.launches - before;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    c->counters.launches = before;
    if (S->gexec) {
      CU(cudaGraphLaunch(S->gexec, st));
      c->counters.launches += S->g_launches;
    } else {
      TRY(omega_sequence(c, S, st));  // capture failed: run the launches directly
    }
  } else {
    TRY(omega_sequence(c, S, st));
  }
  S->g_calls++;
  int hs = 0;
  CU(cudaMemcpyAsync(&hs, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (hs != 0) {
    cudaMemsetAsync(S->status, 0, sizeof(int), st);
    return hs == 2 ? CC3_FAIL(CC3_ERR_ARG, "a contraction plan addressed outside a slice array")
                   : CC3_FAIL(CC3_ERR_TIMEOUT, "split engine wait gave up");
  }
  c->counters.executed_flop = S->executed;
  c->counters.slices = s;
  return CC3_OK;
}

// Autotuner of the split path: times the residual on a strided sample of the
// triple loop (about 32 triples) for each candidate (K steps per vvov tile,
// N tile of the W build), keeps the fastest for this context and for every
// later context of the same (no, nv, slices).  Outputs of the sample runs are
// scratch: cc3_omega_triples clears its accumulators first.
int split_autotune(cc3_ctx *c, cudaStream_t st, int *ks_out, int *nt_out) {
  SplitState *S = nullptr;
  TRY(split_ready(c, &S, st));
  const int nv = c->nv;
  std::vector<int> ks_c = {200, 400, 800};
  std::vector<int> nt_c = {ntile_for(nv)};
  {
    const int nt = (nv + S_NT_MAX - 1) / S_NT_MAX + 1;  // one more N tile
    const int alt = rup((nv + nt - 1) / nt, 16);
    if (alt != nt_c[0] && alt >= 16) nt_c.push_back(alt);
  }
  const std::vector<int> tri_all = c->tri_host;
  const int ntri_all = c->ntri;
  const int stride = std::max(1, ntri_all / 32);
  std::vector<int> sample;
  for (int t = 0; t < ntri_all; t += stride)
    sample.insert(sample.end(), &tri_all[3 * t], &tri_all[3 * t] + 3);
  c->tri_host = sample;
  c->ntri = (int)(sample.size() / 3);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = CC3_OK;
  float best = 1e30f;
  int bks = S->ks_target, bnt = S->nt_w;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = CC3_FAIL(CC3_ERR_CUDA, "autotune events");
  }
  const bool tr = c->trace.on;
  c->trace.on = false;
  for (int nt : nt_c) {
    for (int ks : ks_c) {
      if (rc != CC3_OK) break;
      S->ks_target = ks;
      S->nt_w = nt;
      S->planned = false;
      if ((rc = build_plans(c, S, st)) != CC3_OK) break;
      if ((rc = split_omega(c, st)) != CC3_OK) break;  // warm
      cudaEventRecord(e0, st);
      if ((rc = split_omega(c, st)) != CC3_OK) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = CC3_FAIL(CC3_ERR_CUDA, "autotune timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bks = ks;
        bnt = nt;
      }
    }
  }
  c->trace.on = tr;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->tri_host = tri_all;
  c->ntri = ntri_all;
  S->ks_target = bks;
  S->nt_w = bnt;
  S->planned = false;
  if (rc != CC3_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[TuneKey{c->no, c->nv, S->s}] = {bks, bnt};
  }
  if (ks_out) *ks_out = bks;
  if (nt_out) *nt_out = bnt > 0 ? bnt : ntile_for(nv);
  return CC3_OK;
}

int split_tuning(cc3_ctx *c, int *ks_out, int *nt_out) {
  SplitState *S = state(c);
  int ks = 400, nt = 0;
  if (S) {
    ks = S->ks_target;
    nt = S->nt_w;
  } else {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey{c->no, c->nv, c->slices > 0 ? c->slices : 6});
    if (it != g_tuned.end()) {
      ks = it->second.first;
      nt = it->second.second;
    }
  }
  if (ks_out) *ks_out = ks;
  if (nt_out) *nt_out = nt > 0 ? nt : ntile_for(c->nv);
  return CC3_OK;
}

// Device bytes of the split path's staged slices and workspace (the same
// arithmetic as stage()), for admission control.
size_t split_footprint(int no, int nv, int s, int ntri) {
  const int vp = rup(nv, 16), op = rup(no, 16);
  const long long nv2 = (long long)nv * nv;
  auto sl = [&](long long rows, long long Kp, long long rps) {
    return arr_elems(Kp, rps, rows / rps, s) * sizeof(__nv_bfloat16);
  };
  size_t b = 0;
  b += sl((long long)no * no * nv, vp, nv);           // T2S
  b += 2 * sl((long long)no * nv * nv, op, nv);       // T2C, T2R
  b += 2 * sl((long long)no * nv * nv, vp, nv);       // XS, YS
  b += sl((long long)no * no * nv, op, nv);           // OS
  b += 2 * sl((long long)no * nv, (long long)nv * vp, nv);  // Zg, Zh
  b += sl((long long)no * no * (no + 1), vp, no + 1);  // OO
  b += (size_t)no * no * (no + 1) * nv * sizeof(double);  // its FP64 staging copy
  b += sl((long long)no * no, (long long)nv * vp, 1);  // OV
  const double per_slot = (double)nv2 * nv * 24.0 + 3.0 * s * nv2 * vp * 2.0;
  int batch = (int)std::max(1.0, std::min(16.0, 6.0e9 / per_slot));
  batch = std::min(batch, std::max(1, ntri));
  b += 3 * (size_t)batch * nv2 * nv * sizeof(float2);  // Wdd, TTdd, W3dd
  b += (size_t)std::max(1, ntri) * sizeof(float2);       // eo_tri
  b += 3 * arr_elems((long long)nv * vp, nv, batch, s) * sizeof(__nv_bfloat16);  // V[3]
  b += (size_t)nv * sizeof(float2) + 4096;
  return b;
}

void split_invalidate(cc3_ctx *c) {
  SplitState *S = state(c);
  if (S) S->planned = false;
  // a new triple list changes the batch size; restage lazily
  if (S) {
    split_destroy(c);
  }
}

void split_destroy(cc3_ctx *c) {
  SplitState *S = state(c);
  if (!S) return;
  free_state_buffers(S);
  delete S;
  c->split = nullptr;
}


// ---- right Jacobian transformation (eq. "jcc3", Algorithm 2) -------------------
namespace {

// one slice array from an FP64 tensor through a strided gather (allocates)
int slice_array(SplitState *S, __nv_bfloat16 **dst, const double *src, long long rows, int Kp,
                int E, const Gather &g, int rps, cudaStream_t st) {
  const size_t n = arr_elems(Kp, rps, rows / rps, S->s);
  TRY(alloc(dst, n));
  CU(cudaMemsetAsync(*dst, 0, n * sizeof(__nv_bfloat16), st));
  return launch_slice_gather(src, *dst, S->s, E, g, rows, Kp, rps, st);
}

// ovov in the layouts of Algorithm 2 (once per context):
//   OVD[(q,r)][d][z] = (qd|rz)                  (Z~v: rows d, K = z)
//   OVZA[r][l][(u,w)] = (lu|rw), OVZB[r][l][(u,w)] = (lw|ru)   (Z~o: rows l, K = (zb, u, zz))
int stage_jac_static(cc3_ctx *c, SplitState *S, cudaStream_t st) {
  if (S->OVD) return CC3_OK;
  const int no = c->no, nv = c->nv, vp = S->vp;
  const long long nvo = (long long)nv * no, ovl = (long long)nv * no * nv;
  Gather g;
  g = {0, ovl, nv, nvo, 0, 1, no, nv, vp, nv, 1};
  TRY(slice_array(S, &S->OVD, c->ovov, (long long)no * no * nv, vp, S->Eg, g, nv, st));
  g = {0, 0, nv, ovl, nvo, 1, no, no, nv, nv, nv, 1};
  TRY(slice_array(S, &S->OVZA, c->ovov, (long long)no * no, nv * vp, S->Eg, g, no, st));
  g = {0, 0, nv, ovl, 1, nvo, no, no, nv, nv, nv, 1};
  TRY(slice_array(S, &S->OVZB, c->ovov, (long long)no * no, nv * vp, S->Eg, g, no, st));
  SArr *M = S->arrs.a;
  M[MJ_OVD] = make_arr(S->OVD, vp, nv, (long long)no * no, S->s);
  M[MJ_OVZA] = make_arr(S->OVZA, (long long)nv * vp, no, no, S->s);
  M[MJ_OVZB] = make_arr(S->OVZB, (long long)nv * vp, no, no, S->s);
  return CC3_OK;
}

// Jobs of one distinct permutation (p,q,r) = (ijk[m0], ijk[m1], ijk[m2]) of a
// triple whose tau~ sits in `slot` of the V layouts:
//   F^ term:  rho~_v[p][q][x][y] += sum_z tau~[x][y][z] F^_v[r][z]   (column v)
//   Z~v:      Z~v[x][y][p][d]    -= sum_z tau~[x][y][z] (qd|rz)
//   Z~o:      Z~o[x][q][p][l]    += sum_yz tau~[x][y][z] (ly|rz)
void plan_jac_tau(SPlan *pf, SPlan *pz, SplitState *S, int no, int nv, int nvec, int EF,
                  const int ijk[3], int slot, double &ex) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const int s = S->s, vp = S->vp, nv8 = (nv + 7) / 8 * 8;
  const long long nv2 = (long long)nv * nv, nt2 = (long long)no * no * nv2;
  int seen[6][3], nseen = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int u = 0; u < 6; ++u) {
    const int *m = PERM6[u];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int w = 0; w < nseen; ++w)
      if (seen[w][0] == p && seen[w][1] == q && seen[w][2] == r) dup = true;
    if (dup) continue;
    seen[nseen][0] = p;
    seen[nseen][1] = q;
    seen[nseen][2] = r;
    ++nseen;
    // rows (y_L, x_L) of the z-innermost layout Lz (see plan_omega_split)
    const int Lz = (m[2] + 1) % 3;
    const bool xouter = (m[0] == Lz);
    if (pf) {
      int jb = new_sjob(*pf, nv * nv8, nvec, ntile_for(nvec), 1, 1, SEPI_F64_ATOMIC, EF - 14,
                        ex, s);
      SJob &J = pf->jobs[jb];
      J.expo_slot = slot;
      J.m_pad = nv8;
      J.m_valid = nv;
      OutD c = outd(B_OMT, ((long long)p * no + q) * nv2, xouter ? nv : 1, nt2);
      c.m_in = nv8;
      c.sm1 = xouter ? 1 : nv;
      J.C = c;
      J.Ct = c;
      add_sterm(*pf, jb, opd(MA_V0K + Lz, slot), opd(MJ_FH, r), vp, 0, ex, s);
    }
    if (pz) {
      const long long sx = nv2 * no, sy = (long long)no * nv;  // Z~v strides of x, y
      int jb = new_sjob(*pz, nv * nv8, nv, S->Nab, 1, 1, SEPI_F64_ATOMIC, S->Eg - 14, ex, s);
      SJob &J = pz->jobs[jb];
      J.expo_slot = slot;
      J.m_pad = nv8;
      J.m_valid = nv;
      OutD c = outd(B_ZV, (long long)p * nv, xouter ? sx : sy, 1);
      c.m_in = nv8;
      c.sm1 = xouter ? sy : sx;
      J.C = c;
      J.Ct = c;
      add_sterm(*pz, jb, opd(MA_V0K + Lz, slot), opd(MJ_OVD, q * no + r), vp, 1, ex, s);
      // rows x of layout L = m0, K = (slot L+1, slot L+2) in (zb, u, zz) order
      const int L = m[0];
      const bool yz = (m[1] == (L + 1) % 3);
      jb = new_sjob(*pz, nv, no, ntile_for(no), 1, S->ks4, SEPI_F64_ATOMIC, S->Eg - 14, ex, s);
      SJob &K = pz->jobs[jb];
      K.expo_slot = slot;
      K.C = outd(B_ZO, ((long long)q * no + p) * no, (long long)no * no * no, 1);
      K.Ct = K.C;
      add_sterm(*pz, jb, opd(MA_V0 + L, slot), opd(yz ? MJ_OVZA : MJ_OVZB, r), nv * vp, 0, ex,
                s);
    }
  }
}

struct JacBufs {
  std::vector<void *> p;
  ~JacBufs() {
    for (void *x : p)
      if (x) cudaFree(x);
  }
  template <class T>
  int get(T **out, size_t n) {
    TRY(alloc(out, n));
    p.push_back(*out);
    return CC3_OK;
  }
};

struct JacPlans {
  std::vector<SDevPlan> v;
  ~JacPlans() {
    for (auto &d : v) s_free_plan(&d);
  }
};

}  // namespace

int split_jacobian(cc3_ctx *c, int nvec, const double *w, const double *R1d, const double *R2d,
                   double *rho1d, double *rho2d, cudaStream_t st) {
  SplitState *S = nullptr;
  TRY(split_ready(c, &S, st));
  TRY(jac_blocks(c, st));
  TRY(stage_jac_static(c, S, st));
  const int no = c->no, nv = c->nv, s = S->s, vp = S->vp, op = S->op;
  const long long nv2 = (long long)nv * nv, nvo = (long long)nv * no;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv, nvvvo = (size_t)nv2 * nv * no,
               noovo = (size_t)no * no * nv * no;
  JacBufs B;
  double *hv = nullptr, *ho = nullptr, *hf = nullptr, *mj = nullptr, *rt = nullptr, *r1a = nullptr;
  TRY(B.get(&hv, nvvvo * nvec));
  TRY(B.get(&ho, noovo * nvec));
  TRY(B.get(&hf, n1 * nvec));
  TRY(B.get(&mj, (size_t)c->naux * nv * no));
  TRY(B.get(&rt, nt2 * nvec));
  TRY(B.get(&r1a, n1 * nvec));
  TRY(launch_zero(rt, nt2 * nvec, st));
  TRY(launch_zero(r1a, n1 * nvec, st));
  // R1-dressed integrals of every vector: FP64 engine, except the Cholesky
  // (vvvv) term sum_J L^J_bd M^J_ck of g^_vvvo, a plain nv^2 x nv no x naux
  // contraction done here on the tensor cores
  const int Kj = rup(c->naux, 16);
  if (!S->LVV) {
    const int n = no + nv;
    unsigned long long *ml = nullptr;
    TRY(B.get(&ml, 1));
    CU(cudaMemsetAsync(ml, 0, sizeof(unsigned long long), st));
    TRY(launch_maxabs(c->chol, (long long)c->naux * n * n, ml, st));
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, ml, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double mxl;
    std::memcpy(&mxl, &hb, 8);
    S->EL = exponent_of(mxl);
    const Gather g = {(long long)no * n + no, 0, n, 1, 0, (long long)n * n, nv, nv, Kj, c->naux, 1};
    TRY(slice_array(S, &S->LVV, c->chol, nv2, Kj, S->EL, g, (int)nv2, st));
  }
  {
    __nv_bfloat16 *mjs = nullptr;
    unsigned long long *mm = nullptr;
    TRY(B.get(&mjs, arr_elems(Kj, nvo, 1, s)));
    TRY(B.get(&mm, 1));
    SArrTable la;
    std::memset(&la, 0, sizeof(la));
    la.a[0] = make_arr(S->LVV, Kj, nv2, 1, s);
    la.a[1] = make_arr(mjs, Kj, nvo, 1, s);
    for (int v = 0; v < nvec; ++v) {
      TRY(jac_dress(c, R1d + v * n1, hv + v * nvvvo, ho + v * noovo, hf + v * n1, mj, st, false));
      CU(cudaMemsetAsync(mm, 0, sizeof(unsigned long long), st));
      TRY(launch_maxabs(mj, (long long)c->naux * nvo, mm, st));
      unsigned long long hb = 0;
      CU(cudaMemcpyAsync(&hb, mm, sizeof(hb), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      double mxm;
      std::memcpy(&mxm, &hb, 8);
      if (!(mxm > 0.0)) continue;  // R1 = 0: no vvvv term
      const int EM = exponent_of(mxm);
      CU(cudaMemsetAsync(mjs, 0, arr_elems(Kj, nvo, 1, s) * sizeof(__nv_bfloat16), st));
      const Gather g = {0, 0, no, 1, 0, nvo, nv, no, Kj, c->naux, 1};
      TRY(launch_slice_gather(mj, mjs, s, EM, g, nvo, Kj, (int)nvo, st));
      SPlan P;
      double exc = 0.0;
      const int jb = new_sjob(P, (int)nv2, (int)nvo, ntile_for((int)nvo), 1, 1, SEPI_F64_ATOMIC,
                              S->EL + EM - 14, exc, s);
      P.jobs[jb].C = outd(0, 0, nvo, 1);
      P.jobs[jb].Ct = P.jobs[jb].C;
      add_sterm(P, jb, opd(0, 0), opd(1, 0), Kj, 0, exc, s);
      SDevPlan D;
      TRY(s_upload_plan(P, &D, st));
      VPtrTable vp2;
      std::memset(&vp2, 0, sizeof(vp2));
      vp2.p[0] = hv + v * nvvvo;
      trace_begin(c, TR_SPLIT_W, st);
      const int lrc = s_launch_plan(D, la, vp2, s, S_DRAIN_STEPS, S->status, st,
                                    &c->counters.launches);
      trace_end(c, TR_SPLIT_W, st, D.flop, D.slice_flop);
      CU(cudaStreamSynchronize(st));
      s_free_plan(&D);
      TRY(lrc);
    }
  }
  // exponents: one for all R2 . g and t2 . g^ products, one for F^
  unsigned long long *mx = nullptr;
  TRY(B.get(&mx, 2 * (size_t)nvec + 1));
  CU(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (2 * nvec + 1), st));
  for (int v = 0; v < nvec; ++v) {
    TRY(launch_maxabs(R2d + v * nt2, (long long)nt2, mx + v, st));
    TRY(launch_maxabs(hv + v * nvvvo, (long long)nvvvo, mx + nvec + v, st));
    TRY(launch_maxabs(ho + v * noovo, (long long)noovo, mx + nvec + v, st));
  }
  TRY(launch_maxabs(hf, (long long)n1 * nvec, mx + 2 * nvec, st));
  std::vector<unsigned long long> hm(2 * nvec + 1);
  CU(cudaMemcpyAsync(hm.data(), mx, sizeof(unsigned long long) * hm.size(),
                     cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  auto ex_of = [&](int i, int dflt) {
    double x;
    std::memcpy(&x, &hm[i], 8);
    return x > 0.0 ? exponent_of(x) : dflt;
  };
  int Ec = -100000;
  for (int v = 0; v < nvec; ++v) {
    Ec = std::max(Ec, ex_of(v, -100000) + S->Eg);
    Ec = std::max(Ec, S->Et + ex_of(nvec + v, -100000));
  }
  if (Ec < -50000) Ec = S->Et + S->Eg;  // R2 = 0 and R1 = 0: the result is 0
  const int ER = Ec - S->Eg, EH = Ec - S->Et, EF = ex_of(2 * nvec, 0);
  // slices of R2 (t2 layouts), g^ (vvvo / oovo layouts) and F^; each kind holds
  // the slices of every vector back to back (vector v's slabs follow v - 1's)
  const long long oo = (long long)no * no, onv = (long long)no * nv;
  struct Kind {
    int map;
    long long K, rps, slabs;  // K, rows per slab, slabs per vector
    __nv_bfloat16 *base;
  };
  Kind kinds[6] = {{MJ_R2S, vp, nv, oo, nullptr},  {MJ_R2C, op, nv, onv, nullptr},
                   {MJ_R2R, op, nv, onv, nullptr}, {MJ_XH, vp, nv, onv, nullptr},
                   {MJ_YH, vp, nv, onv, nullptr},  {MJ_OH, op, nv, oo, nullptr}};
  SArrTable jr = S->arrs;  // the R3 part: combined vector arrays, R3 slot arrays
  for (Kind &k : kinds) {
    const size_t per = arr_elems(k.K, k.rps, k.slabs, s);
    TRY(B.get(&k.base, per * nvec));
    CU(cudaMemsetAsync(k.base, 0, per * nvec * sizeof(__nv_bfloat16), st));
    jr.a[k.map] = make_arr(k.base, k.K, k.rps, k.slabs * nvec, s);
  }
  for (int v = 0; v < nvec; ++v) {
    const double *r2 = R2d + v * nt2, *gv = hv + v * nvvvo, *go = ho + v * noovo;
    auto dst = [&](int i) {
      return kinds[i].base + (size_t)v * arr_elems(kinds[i].K, kinds[i].rps, kinds[i].slabs, s);
    };
    Gather g;
    g = {0, (long long)no * nv2, nv2, nv, 0, 1, no, nv, vp, nv, 1};
    TRY(launch_slice_gather(r2, dst(0), s, ER, g, oo * nv, vp, nv, st));
    g = {0, (long long)no * nv2, 1, nv, 0, nv2, nv, nv, op, no, 1};
    TRY(launch_slice_gather(r2, dst(1), s, ER, g, onv * nv, op, nv, st));
    g = {0, (long long)no * nv2, nv, 1, 0, nv2, nv, nv, op, no, 1};
    TRY(launch_slice_gather(r2, dst(2), s, ER, g, onv * nv, op, nv, st));
    g = {0, 1, no, nv2 * no, 0, nvo, nv, nv, vp, nv, 1};
    TRY(launch_slice_gather(gv, dst(3), s, EH, g, onv * nv, vp, nv, st));
    g = {0, 1, nv2 * no, no, 0, nvo, nv, nv, vp, nv, 1};
    TRY(launch_slice_gather(gv, dst(4), s, EH, g, onv * nv, vp, nv, st));
    g = {0, nvo, 1, no, 0, (long long)no * nv * no, no, nv, op, no, 1};
    TRY(launch_slice_gather(go, dst(5), s, EH, g, oo * nv, op, nv, st));
  }
  {
    __nv_bfloat16 *a = nullptr;
    Gather g = {0, 0, nv, nvo, 0, 1, no, nvec, vp, nv, 1};
    TRY(slice_array(S, &a, hf, (long long)no * nvec, vp, EF, g, nvec, st));
    B.p.push_back(a);
    S->arrs.a[MJ_FH] = jr.a[MJ_FH] = make_arr(a, vp, nvec, no, s);
  }
  // Batches: bj triples share tau~3 (the residual's workspace); the R3 of all
  // vectors for those triples fill nvec * bj slots of a workspace of their
  // own, slot u = v * bj + t, so that each phase is one launch per batch
  // whatever the number of vectors.
  const double per_slot = (double)nv2 * nv * 24.0 + 3.0 * s * nv2 * vp * 2.0;
  const int bj = std::max(1, std::min(S->batch, (int)(12.0e9 / (per_slot * nvec))));
  const int nslot = nvec * bj;
  float2 *Wj = nullptr, *TTj = nullptr, *W3j = nullptr, *eoj = nullptr;
  __nv_bfloat16 *Vj[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16 **vptrj = nullptr;
  unsigned int *maxj = nullptr;
  int *exj = nullptr;
  TRY(B.get(&Wj, (size_t)nslot * nv2 * nv));
  TRY(B.get(&TTj, (size_t)nslot * nv2 * nv));
  TRY(B.get(&W3j, (size_t)nslot * nv2 * nv));
  TRY(B.get(&eoj, (size_t)nslot));
  TRY(B.get(&maxj, (size_t)nslot));
  TRY(B.get(&exj, (size_t)nslot));
  TRY(B.get(&vptrj, 3));
  const long long nv8 = (nv + 7) / 8 * 8;
  for (int L = 0; L < 3; ++L) {
    const size_t n4 = arr_elems((long long)nv * vp, nv, nslot, s);
    TRY(B.get(&Vj[L], n4));
    CU(cudaMemsetAsync(Vj[L], 0, n4 * sizeof(__nv_bfloat16), st));
    jr.a[MA_V0 + L] = make_arr(Vj[L], (long long)nv * vp, nv, nslot, s);
    jr.a[MA_V0K + L] = make_arr(Vj[L], vp, (long long)nv * nv8, nslot, s);
  }
  CU(cudaMemcpyAsync(vptrj, Vj, sizeof(Vj), cudaMemcpyHostToDevice, st));
  // plans per batch: tau3's W build, the tau~ . F^ jobs and, when the cache is
  // cold, Z~v, Z~o (slots t); the R3 W build and contractions of all vectors
  // (slots u, outputs offset to each vector's rho~)
  const bool prep = jac_prep_prec(c) < 0;
  double *Zv = nullptr, *Zo = nullptr;
  TRY(jac_z_buffers(c, &Zv, &Zo, prep, st));
  const int rows = (nv + 7) / 8 * 8;
  const int ks4 = S->ks4;
  const bool stack = S->stack_vvov && nv >= S_BM && nv % 8 == 0 && nv % S_BM != 0;
  const int nb = (c->ntri + bj - 1) / bj;
  JacPlans pT, pAB, pF, pZ, pO;
  pT.v.resize(nb);
  pAB.v.resize(nb);
  pF.v.resize(nb);
  pZ.v.resize(nb);
  pO.v.resize(nb);
  std::vector<float2> eoh((size_t)nslot * nb);
  double ex = 0.0, ex_tau = 0.0;
  for (int b = 0; b < nb; ++b) {
    const int t0 = b * bj, t1 = std::min(c->ntri, t0 + bj);
    SPlan tb, ab, f, z, om, om3;
    std::vector<VvovPerm> vperms;
    for (int t = t0; t < t1; ++t) {
      const int *ijk = &c->tri_host[3 * t];
      plan_w_split(tb, S, no, nv, ijk, t - t0, ex_tau);
      plan_jac_tau(&f, prep ? &z : nullptr, S, no, nv, nvec, EF, ijk, t - t0, ex);
      const double eo_sum = c->eo_h[ijk[0]] + c->eo_h[ijk[1]] + c->eo_h[ijk[2]];
      for (int v = 0; v < nvec; ++v) {
        const int u = v * bj + (t - t0);
        // the element-wise step divides by (0 - (e_a+e_b+e_c - eo)): with
        // eo = e_i + e_j + e_k + w that is (w - eps)
        const dd::df e = dd::from_double_host(eo_sum + w[v]);
        eoh[(size_t)b * nslot + u] = make_float2(e.hi, e.lo);
        WMaps set1 = {MJ_R2S, MJ_R2S, MJ_R2C, MJ_R2C, MJ_R2R, MJ_R2R,
                      MA_XS,  MB_XS,  MA_YS,  MB_YS,  MA_OS,  MB_OS};
        set1.oS = (int)(v * oo);
        set1.oC = set1.oR = (int)(v * onv);
        WMaps set2 = {MA_T2S, MB_T2S, MA_T2C, MB_T2C, MA_T2R, MB_T2R,
                      MJ_XH,  MJ_XH,  MJ_YH,  MJ_YH,  MJ_OH,  MJ_OH};
        set2.oXS = set2.oYS = (int)(v * onv);
        set2.oOS = (int)(v * oo);
        const int j1 = w_job(ab, nv, rows, S->Nab, 1, u, Ec - 14, ex, s);
        w_terms_1(ab, j1, set1, no, nv, rows, vp, op, ijk, ex, s);
        w_terms_1(ab, j1, set2, no, nv, rows, vp, op, ijk, ex, s);
        const int j2 = w_job(ab, nv, rows, S->Nab, 2, u, Ec - 14, ex, s);
        w_terms_2(ab, j2, set1, no, nv, rows, vp, op, ijk, ex, s);
        w_terms_2(ab, j2, set2, no, nv, rows, vp, op, ijk, ex, s);
        const int j3 = w_job(ab, nv, rows, S->Nab, 3, u, Ec - 14, ex, s);
        w_terms_3(ab, j3, set1, no, nv, rows, vp, op, ijk, ex, s);
        w_terms_3(ab, j3, set2, no, nv, rows, vp, op, ijk, ex, s);
        // the contractions of R~3 into vector v's rho~ and rho1
        const size_t first = om3.jobs.size();
        if (stack) {
          const size_t f0 = vperms.size();
          collect_vvov_perms(vperms, ijk, u);
          for (size_t k = f0; k < vperms.size(); ++k) {
            vperms[k].omt_off = (long long)v * nt2;
            vperms[k].om1_off = (long long)v * n1;
          }
        } else {
          plan_omega_split(om3, S, no, nv, ijk, u, ks4, ex, 1);
        }
        plan_omega_split(om3, S, no, nv, ijk, u, ks4, ex, 2);
        for (size_t jx = first; jx < om3.jobs.size(); ++jx) {
          SJob &J = om3.jobs[jx];
          for (OutD *o : {&J.C, &J.Ct, &J.C2, &J.Ct2}) {
            if (o->buf == B_OMT) o->off += (long long)v * nt2;
            else if (o->buf == B_OM1) o->off += (long long)v * n1;
          }
        }
      }
    }
    if (stack) plan_vvov_stacked(om, S, no, nv, vperms, ks4, ex);
    append_plan(om, om3);  // the long-K vvov tiles first
    TRY(s_upload_plan(tb, &pT.v[b], st));
    TRY(s_upload_plan(ab, &pAB.v[b], st));
    TRY(s_upload_plan(f, &pF.v[b], st));
    if (prep) TRY(s_upload_plan(z, &pZ.v[b], st));
    TRY(s_upload_plan(om, &pO.v[b], st));
  }
  float2 *eoj_all = nullptr;
  TRY(B.get(&eoj_all, eoh.size()));
  CU(cudaMemcpyAsync(eoj_all, eoh.data(), sizeof(float2) * eoh.size(), cudaMemcpyHostToDevice,
                     st));
  // the loop: per batch, tau~3 and its jobs, then the R3 of every vector
  VPtrTable P;
  fill_vptrs(c, S, &P);
  P.p[B_ZV] = Zv;
  P.p[B_ZO] = Zo;
  P.p[B_OMT] = rt;
  P.p[B_OM1] = r1a;
  VPtrTable PR = P;
  PR.p[B_WS_W] = Wj;
  PR.p[B_WS_TT] = TTj;
  PR.p[B_WS_W3] = W3j;
  PR.p[B_SLOTEXP] = exj;
  const int kd = S_DRAIN_STEPS;
  long long *L = &c->counters.launches;
  auto run = [&](const SDevPlan &d, const SArrTable &a, const VPtrTable &pt, int cls) -> int {
    trace_begin(c, cls, st);
    TRY(s_launch_plan(d, a, pt, s, kd, S->status, st, L));
    trace_end(c, cls, st, d.flop, d.slice_flop);
    return CC3_OK;
  };
  // tau (or R3) and tau~ from the W build's partial sums, slot exponents and
  // the slices of the contravariant amplitudes
  auto elem = [&](float2 *W1, float2 *W2, float2 *W3, const float2 *eo, int ns,
                  unsigned int *mb, int *exs, __nv_bfloat16 **vp_dev, int nalloc) -> int {
    trace_begin(c, TR_SPLIT_ELEM, st);
    CU(cudaMemsetAsync(mb, 0, sizeof(unsigned int) * ns, st));
    TRY(launch_tau_contravariant_dd(W1, W2, W3, W2, S->evdd, eo, 0.f, 0.f, nv, ns, mb, st));
    TRY(launch_slot_exponent(mb, exs, ns, st));
    TRY(launch_slice_tt(W2, vp_dev, nv, vp, s, exs, ns, nalloc, st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    *L += 3;
    return CC3_OK;
  };
  for (int b = 0; b < nb; ++b) {
    const int t0 = b * bj, ns = std::min(c->ntri, t0 + bj) - t0;
    TRY(run(pT.v[b], S->arrs, P, TR_SPLIT_W));
    TRY(elem(S->Wdd, S->TTdd, S->W3dd, S->eo_tri + t0, ns, S->maxbits, S->slot_ex, S->vptr,
             S->batch));
    if (prep) TRY(run(pZ.v[b], S->arrs, P, TR_SPLIT_OMEGA));
    TRY(run(pF.v[b], S->arrs, P, TR_SPLIT_OMEGA));
    TRY(run(pAB.v[b], jr, PR, TR_SPLIT_W));
    TRY(elem(Wj, TTj, W3j, eoj_all + (size_t)b * nslot, nslot, maxj, exj, vptrj, nslot));
    TRY(run(pO.v[b], jr, PR, TR_SPLIT_OMEGA));
  }
  int hs = 0;
  CU(cudaMemcpyAsync(&hs, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (hs != 0) {
    cudaMemsetAsync(S->status, 0, sizeof(int), st);
    return hs == 2 ? CC3_FAIL(CC3_ERR_ARG, "a Jacobian plan addressed outside a slice array")
                   : CC3_FAIL(CC3_ERR_TIMEOUT, "split engine wait gave up");
  }
  if (prep) jac_set_prep(c, CC3_SPLIT_BF16);
  // Z~ . R1 (FP64), back-transform, singles
  for (int v = 0; v < nvec; ++v) {
    TRY(jac_z_terms(c, R1d + v * n1, rt + v * nt2, st));
    TRY(launch_back_transform(rt + v * nt2, rho2d + v * nt2, no, nv, st));
    CU(cudaMemcpyAsync(rho1d + v * n1, r1a + v * n1, sizeof(double) * n1,
                       cudaMemcpyDeviceToDevice, st));
  }
  CU(cudaStreamSynchronize(st));
  c->counters.executed_flop = ex + ex_tau;
  c->counters.slices = s;
  return CC3_OK;
}

// ---- left (transpose) Jacobian transformation -----------------------------------
namespace {

// One permutation's term of the G contraction (see plan_left_g).
struct GTerm {
  int v, r, mi, u, p, q;
};

// Jobs of the left transformation for one triple (every distinct permutation
// (p,q,r) = (ijk[m0], ijk[m1], ijk[m2]); layouts as in plan_jac_tau):
//   pgh, on L~3 in slot u of vector v (H at the vector's offset hoff; the G
//   terms go to gterms, made into jobs by plan_left_g):
//     H[l][q][z][r] += sum_xy L~[x][y][z] t[p][l][x][y]  rows z of layout m2, K = (zb, u, zz)
//   pq, on tau~3 in slot u (all vectors at once, column v):
//     Q[v][r][z]    += sum_xy Lt2_v[p][q][x][y] tau~[x][y][z]
void plan_left_split(SPlan *pgh, SPlan *pq, std::vector<GTerm> *gterms, SplitState *S, int no,
                     int nv, int ELt, int nvec, const int ijk[3], int u, int v, long long hoff,
                     double &ex) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const int s = S->s, vp = S->vp;
  const long long nvo = (long long)nv * no, n1 = nvo;
  int seen[6][3], nseen = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int w = 0; w < 6; ++w) {
    const int *m = PERM6[w];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int x = 0; x < nseen; ++x)
      if (seen[x][0] == p && seen[x][1] == q && seen[x][2] == r) dup = true;
    if (dup) continue;
    seen[nseen][0] = p;
    seen[nseen][1] = q;
    seen[nseen][2] = r;
    ++nseen;
    const int Lz = m[2];                          // rows z, K over the other two slots
    const bool yz = (m[0] == (Lz + 1) % 3);       // K = (zb over y, x, zz) or (.., y, ..)
    if (gterms) gterms->push_back(GTerm{v, r, w, u, p, q});
    if (pgh) {
      int jb = new_sjob(*pgh, nv, no, ntile_for(no), 1, S->ks4, SEPI_F64_ATOMIC, S->Et - 14, ex, s);
      SJob &K = pgh->jobs[jb];
      K.expo_slot = u;
      K.C = outd(B_H, hoff + (long long)q * nvo + r, no, (long long)no * nvo);
      K.Ct = K.C;
      add_sterm(*pgh, jb, opd(MA_V0 + Lz, u), opd(yz ? ML_T2ZA : ML_T2ZB, p), nv * vp, 0, ex, s);
    }
    if (pq) {
      int jb = new_sjob(*pq, nv, nvec, ntile_for(nvec), 1, S->ks4, SEPI_F64_ATOMIC, ELt - 14,
                        ex, s);
      SJob &J = pq->jobs[jb];
      J.expo_slot = u;
      J.C = outd(B_Q, (long long)r * nv, 1, n1);
      J.Ct = J.C;
      add_sterm(*pq, jb, opd(MA_V0 + Lz, u), opd(yz ? ML_LQA : ML_LQB, p * no + q), nv * vp, 0,
                ex, s);
    }
  }
}

// The G contraction of a batch, G[y][d][z][r] += sum_x L~[x][y][z] t[p][q][x][d],
// rows (y_L, x_L) of layout (m0+1)%3, K = x: the permutations of the batch with the
// same vector, output index r and slot map m write the same output rows in the
// same order, so they become the terms of one job (K = their number times nv).
// All L3 slots of a batch share one exponent, so the job's scale is that of any.
void plan_left_g(SPlan &P, SplitState *S, int no, int nv, std::vector<GTerm> terms,
                 size_t ng, double &ex) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const int s = S->s, vp = S->vp, nv8 = (nv + 7) / 8 * 8;
  const long long nv2 = (long long)nv * nv, nvo = (long long)nv * no;
  std::stable_sort(terms.begin(), terms.end(), [](const GTerm &a, const GTerm &b) {
    return a.v != b.v ? a.v < b.v : (a.r != b.r ? a.r < b.r : a.mi < b.mi);
  });
  for (size_t g0 = 0; g0 < terms.size();) {
    size_t g1 = g0 + 1;
    while (g1 < terms.size() && terms[g1].v == terms[g0].v && terms[g1].r == terms[g0].r &&
           terms[g1].mi == terms[g0].mi)
      ++g1;
    const GTerm &f = terms[g0];
    const int *m = PERM6[f.mi];
    const int L = (m[0] + 1) % 3;  // K = slot L+2 = x; rows (slot L+1, slot L)
    const bool xl_y = (L == m[1]);
    const int ksteps = (int)(g1 - g0) * (vp / 16);
    const int ksplit = std::max(1, std::min(8, ksteps / 192));
    int jb = new_sjob(P, nv * nv8, nv, ntile_for(nv), 1, ksplit, SEPI_F64_ATOMIC, S->Et - 14,
                      ex, s);
    SJob &J = P.jobs[jb];
    J.expo_slot = f.u;
    J.m_pad = nv8;
    J.m_valid = nv;
    OutD c = outd(B_G, (long long)f.v * (long long)ng + f.r, xl_y ? nv2 * no : no, nvo);
    c.m_in = nv8;
    c.sm1 = xl_y ? no : nv2 * no;
    J.C = c;
    J.Ct = c;
    for (size_t k = g0; k < g1; ++k)
      add_sterm(P, jb, opd(MA_V0K + L, terms[k].u), opd(ML_T2T, terms[k].p * no + terms[k].q),
                vp, 0, ex, s);
    g0 = g1;
  }
}

}  // namespace

// The left transformation on the tensor cores.  Per batch of triples: tau3
// (the residual's W build and element-wise step) with the Algorithm 2 jobs
// when the cache is cold and the Q jobs of every vector; then the L3 of every
// vector (slots u = v * bj + t): the W-build bracket of Lt2 on the engine, the
// outer products L1 (x) g_ovov + Lt2 (x) F in double-float, the element-wise
// step with (w - eps), and the contractions of L~3 (the residual's vvov and
// ooov ones without the singles and F columns into sigma2, and G, H).  sigma1
// then follows in FP64 from Q, G, H, Lt2 and the Algorithm 2 intermediates,
// as on the FP64 path.
int split_left_jacobian(cc3_ctx *c, int nvec, const double *w, const double *L1d,
                        const double *L2d, double *s1d, double *s2d, cudaStream_t st) {
  SplitState *S = nullptr;
  TRY(split_ready(c, &S, st));
  TRY(jac_blocks(c, st));
  TRY(stage_jac_static(c, S, st));
  const int no = c->no, nv = c->nv, s = S->s, vp = S->vp, op = S->op;
  const long long nv2 = (long long)nv * nv, oo = (long long)no * no;
  const long long onv = (long long)no * nv;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv, ng = (size_t)nv2 * nv * no,
               nh = (size_t)no * no * nv * no;
  JacBufs B;
  double *lt = nullptr, *s2raw = nullptr, *Q = nullptr, *G = nullptr, *H = nullptr,
         *N = nullptr;
  float2 *l1dd = nullptr, *ltdd = nullptr, *ovdd = nullptr, *fdd = nullptr;
  int *tri_all = nullptr;
  TRY(B.get(&lt, nt2 * nvec));
  TRY(B.get(&s2raw, nt2 * nvec));
  TRY(B.get(&Q, n1 * nvec));
  TRY(B.get(&G, ng * nvec));
  TRY(B.get(&H, nh * nvec));
  TRY(B.get(&N, (size_t)c->naux * nv * no));
  TRY(B.get(&l1dd, n1 * nvec));
  TRY(B.get(&ltdd, nt2 * nvec));
  TRY(B.get(&ovdd, (size_t)(oo * nv2)));
  TRY(B.get(&fdd, n1));
  TRY(B.get(&tri_all, 3 * (size_t)c->ntri));
  CU(cudaMemcpyAsync(tri_all, c->tri_host.data(), sizeof(int) * 3 * c->ntri,
                     cudaMemcpyHostToDevice, st));
  TRY(launch_zero(s2raw, nt2 * nvec, st));
  TRY(launch_zero(Q, n1 * nvec, st));
  TRY(launch_zero(G, ng * nvec, st));
  TRY(launch_zero(H, nh * nvec, st));
  for (int v = 0; v < nvec; ++v)
    TRY(launch_back_transform(L2d + v * nt2, lt + v * nt2, no, nv, st));
  TRY(launch_to_dd(L1d, l1dd, (long long)(n1 * nvec), st));
  TRY(launch_to_dd(lt, ltdd, (long long)(nt2 * nvec), st));
  TRY(launch_to_dd(c->ovov, ovdd, oo * nv2, st));
  TRY(launch_to_dd(c->F_ov, fdd, (long long)n1, st));
  // one exponent for the slices of Lt2 (all vectors)
  int ELt = 0;
  {
    unsigned long long *mx = nullptr;
    TRY(B.get(&mx, 1));
    CU(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    TRY(launch_maxabs(lt, (long long)(nt2 * nvec), mx, st));
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, mx, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double x;
    std::memcpy(&x, &hb, 8);
    ELt = x > 0.0 ? exponent_of(x) : 0;
  }
  auto sliced = [&](__nv_bfloat16 **dst, const double *src, long long rows, int Kp, int E,
                    const Gather &g, int rps) -> int {
    const size_t n = arr_elems(Kp, rps, rows / rps, s);
    TRY(B.get(dst, n));
    CU(cudaMemsetAsync(*dst, 0, n * sizeof(__nv_bfloat16), st));
    return launch_slice_gather(src, *dst, s, E, g, rows, Kp, rps, st);
  };
  SArrTable jr = S->arrs;  // the L3 part
  SArrTable aq = S->arrs;  // the tau3 part (Q jobs)
  {
    // t2 for G: [(p,q)][d][x];  for H: [p][l][(u,w)], (u,w) = (x,y) or (y,x)
    __nv_bfloat16 *t2t = nullptr, *tza = nullptr, *tzb = nullptr, *lqa = nullptr, *lqb = nullptr;
    Gather g;
    g = {0, (long long)no * nv2, nv2, 1, 0, nv, no, nv, vp, nv, 1, 0};
    TRY(sliced(&t2t, c->t2, oo * nv, vp, S->Et, g, nv));
    g = {0, 0, (long long)no * nv2, nv2, nv, 1, no, no, nv, nv, nv, 1};
    TRY(sliced(&tza, c->t2, oo, nv * vp, S->Et, g, no));
    g = {0, 0, (long long)no * nv2, nv2, 1, nv, no, no, nv, nv, nv, 1};
    TRY(sliced(&tzb, c->t2, oo, nv * vp, S->Et, g, no));
    // Lt2 of every vector: rows v of slab (p,q)
    g = {0, nv2, 0, (long long)nt2, nv, 1, 1, nvec, nv, nv, nv, 1};
    TRY(sliced(&lqa, lt, oo * nvec, nv * vp, ELt, g, nvec));
    g = {0, nv2, 0, (long long)nt2, 1, nv, 1, nvec, nv, nv, nv, 1};
    TRY(sliced(&lqb, lt, oo * nvec, nv * vp, ELt, g, nvec));
    jr.a[ML_T2T] = make_arr(t2t, vp, nv, oo, s);
    jr.a[ML_T2ZA] = make_arr(tza, (long long)nv * vp, no, no, s);
    jr.a[ML_T2ZB] = make_arr(tzb, (long long)nv * vp, no, no, s);
    aq.a[ML_LQA] = make_arr(lqa, (long long)nv * vp, nvec, oo, s);
    aq.a[ML_LQB] = make_arr(lqb, (long long)nv * vp, nvec, oo, s);
  }
  // Lt2 in the t2 roles of the W build (every vector back to back)
  struct Kind {
    int map;
    long long K, rps, slabs;
    __nv_bfloat16 *base;
  };
  Kind kinds[3] = {{MJ_R2S, vp, nv, oo, nullptr}, {MJ_R2C, op, nv, onv, nullptr},
                   {MJ_R2R, op, nv, onv, nullptr}};
  for (Kind &k : kinds) {
    const size_t per = arr_elems(k.K, k.rps, k.slabs, s);
    TRY(B.get(&k.base, per * nvec));
    CU(cudaMemsetAsync(k.base, 0, per * nvec * sizeof(__nv_bfloat16), st));
    jr.a[k.map] = make_arr(k.base, k.K, k.rps, k.slabs * nvec, s);
  }
  for (int v = 0; v < nvec; ++v) {
    const double *l2 = lt + v * nt2;
    auto dst = [&](int i) {
      return kinds[i].base + (size_t)v * arr_elems(kinds[i].K, kinds[i].rps, kinds[i].slabs, s);
    };
    Gather g;
    g = {0, (long long)no * nv2, nv2, nv, 0, 1, no, nv, vp, nv, 1, 0};
    TRY(launch_slice_gather(l2, dst(0), s, ELt, g, oo * nv, vp, nv, st));
    g = {0, (long long)no * nv2, 1, nv, 0, nv2, nv, nv, op, no, 1, 0};
    TRY(launch_slice_gather(l2, dst(1), s, ELt, g, onv * nv, op, nv, st));
    g = {0, (long long)no * nv2, nv, 1, 0, nv2, nv, nv, op, no, 1, 0};
    TRY(launch_slice_gather(l2, dst(2), s, ELt, g, onv * nv, op, nv, st));
  }
  // L3 slots of all vectors (as the right transformation's R3 slots); larger
  // batches than the right transformation's (up to 120 GB, at most 40 % of the free
  // memory) give the grouped G jobs more terms
  const double per_slot = (double)nv2 * nv * 24.0 + 3.0 * s * nv2 * vp * 2.0;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const double slot_budget = std::min(120.0e9, 0.4 * (double)free_b);
  const int bj = std::max(1, std::min(S->batch, (int)(slot_budget / (per_slot * nvec))));
  const int nslot = nvec * bj;
  float2 *Wj = nullptr, *TTj = nullptr, *W3j = nullptr;
  __nv_bfloat16 *Vj[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16 **vptrj = nullptr;
  unsigned int *maxj = nullptr;
  int *exj = nullptr;
  TRY(B.get(&Wj, (size_t)nslot * nv2 * nv));
  TRY(B.get(&TTj, (size_t)nslot * nv2 * nv));
  TRY(B.get(&W3j, (size_t)nslot * nv2 * nv));
  TRY(B.get(&maxj, (size_t)nslot));
  TRY(B.get(&exj, (size_t)nslot));
  TRY(B.get(&vptrj, 3));
  const long long nv8 = (nv + 7) / 8 * 8;
  for (int L = 0; L < 3; ++L) {
    const size_t n4 = arr_elems((long long)nv * vp, nv, nslot, s);
    TRY(B.get(&Vj[L], n4));
    CU(cudaMemsetAsync(Vj[L], 0, n4 * sizeof(__nv_bfloat16), st));
    jr.a[MA_V0 + L] = make_arr(Vj[L], (long long)nv * vp, nv, nslot, s);
    jr.a[MA_V0K + L] = make_arr(Vj[L], vp, (long long)nv * nv8, nslot, s);
  }
  CU(cudaMemcpyAsync(vptrj, Vj, sizeof(Vj), cudaMemcpyHostToDevice, st));
  const bool prep = jac_prep_prec(c) < 0;
  double *Zv = nullptr, *Zo = nullptr;
  TRY(jac_z_buffers(c, &Zv, &Zo, prep, st));
  const int rows = (nv + 7) / 8 * 8;
  const int ks4 = S->ks4;
  const int Ec = ELt + S->Eg;
  const int nb = (c->ntri + bj - 1) / bj;
  JacPlans pT, pZ, pQ, pAB, pO;
  pT.v.resize(nb);
  pZ.v.resize(nb);
  pQ.v.resize(nb);
  pAB.v.resize(nb);
  pO.v.resize(nb);
  std::vector<float2> eoh((size_t)nslot * nb);
  double ex = 0.0, ex_tau = 0.0;
  for (int b = 0; b < nb; ++b) {
    const int t0 = b * bj, t1 = std::min(c->ntri, t0 + bj);
    SPlan tb, z, qp, ab, om;
    std::vector<GTerm> gterms;
    for (int t = t0; t < t1; ++t) {
      const int *ijk = &c->tri_host[3 * t];
      plan_w_split(tb, S, no, nv, ijk, t - t0, ex_tau);
      if (prep) plan_jac_tau(nullptr, &z, S, no, nv, nvec, 0, ijk, t - t0, ex);
      plan_left_split(nullptr, &qp, nullptr, S, no, nv, ELt, nvec, ijk, t - t0, 0, 0, ex);
      const double eo_sum = c->eo_h[ijk[0]] + c->eo_h[ijk[1]] + c->eo_h[ijk[2]];
      for (int v = 0; v < nvec; ++v) {
        const int u = v * bj + (t - t0);
        const dd::df e = dd::from_double_host(eo_sum + w[v]);
        eoh[(size_t)b * nslot + u] = make_float2(e.hi, e.lo);
        WMaps set1 = {MJ_R2S, MJ_R2S, MJ_R2C, MJ_R2C, MJ_R2R, MJ_R2R,
                      MA_XS,  MB_XS,  MA_YS,  MB_YS,  MA_OS,  MB_OS};
        set1.oS = (int)(v * oo);
        set1.oC = set1.oR = (int)(v * onv);
        const int j1 = w_job(ab, nv, rows, S->Nab, 1, u, Ec - 14, ex, s);
        w_terms_1(ab, j1, set1, no, nv, rows, vp, op, ijk, ex, s);
        const int j2 = w_job(ab, nv, rows, S->Nab, 2, u, Ec - 14, ex, s);
        w_terms_2(ab, j2, set1, no, nv, rows, vp, op, ijk, ex, s);
        const int j3 = w_job(ab, nv, rows, S->Nab, 3, u, Ec - 14, ex, s);
        w_terms_3(ab, j3, set1, no, nv, rows, vp, op, ijk, ex, s);
        // sigma2 (the residual's vvov and ooov contractions, no singles or F
        // columns), G and H of vector v
        const size_t first = om.jobs.size();
        plan_omega_split(om, S, no, nv, ijk, u, ks4, ex, 1 | 8);
        plan_omega_split(om, S, no, nv, ijk, u, ks4, ex, 2 | 8);
        for (size_t jx = first; jx < om.jobs.size(); ++jx) {
          SJob &J = om.jobs[jx];
          for (OutD *o : {&J.C, &J.Ct, &J.C2, &J.Ct2})
            if (o->buf == B_OMT) o->off += (long long)v * nt2;
        }
        plan_left_split(&om, nullptr, &gterms, S, no, nv, ELt, nvec, ijk, u, v,
                        (long long)v * nh, ex);
      }
    }
    plan_left_g(om, S, no, nv, gterms, ng, ex);
    TRY(s_upload_plan(tb, &pT.v[b], st));
    if (prep) TRY(s_upload_plan(z, &pZ.v[b], st));
    TRY(s_upload_plan(qp, &pQ.v[b], st));
    TRY(s_upload_plan(ab, &pAB.v[b], st));
    TRY(s_upload_plan(om, &pO.v[b], st));
  }
  float2 *eoj_all = nullptr;
  TRY(B.get(&eoj_all, eoh.size()));
  CU(cudaMemcpyAsync(eoj_all, eoh.data(), sizeof(float2) * eoh.size(), cudaMemcpyHostToDevice,
                     st));
  VPtrTable P;
  fill_vptrs(c, S, &P);
  P.p[B_ZV] = Zv;
  P.p[B_ZO] = Zo;
  P.p[B_Q] = Q;
  VPtrTable PR = P;
  PR.p[B_WS_W] = Wj;
  PR.p[B_WS_TT] = TTj;
  PR.p[B_WS_W3] = W3j;
  PR.p[B_SLOTEXP] = exj;
  PR.p[B_OMT] = s2raw;
  PR.p[B_G] = G;
  PR.p[B_H] = H;
  const int kd = S_DRAIN_STEPS;
  long long *L = &c->counters.launches;
  auto run = [&](const SDevPlan &d, const SArrTable &a, const VPtrTable &pt, int cls) -> int {
    trace_begin(c, cls, st);
    TRY(s_launch_plan(d, a, pt, s, kd, S->status, st, L));
    trace_end(c, cls, st, d.flop, d.slice_flop);
    return CC3_OK;
  };
  auto elem = [&](float2 *W1, float2 *W2, float2 *W3, const float2 *eo, int ns, unsigned int *mb,
                  int *exs, __nv_bfloat16 **vp_dev, int nalloc) -> int {
    trace_begin(c, TR_SPLIT_ELEM, st);
    CU(cudaMemsetAsync(mb, 0, sizeof(unsigned int) * ns, st));
    TRY(launch_tau_contravariant_dd(W1, W2, W3, W2, S->evdd, eo, 0.f, 0.f, nv, ns, mb, st));
    TRY(launch_slot_exponent(mb, exs, ns, st));
    TRY(launch_slice_tt(W2, vp_dev, nv, vp, s, exs, ns, nalloc, st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    *L += 3;
    return CC3_OK;
  };
  for (int b = 0; b < nb; ++b) {
    const int t0 = b * bj, ns = std::min(c->ntri, t0 + bj) - t0;
    TRY(run(pT.v[b], S->arrs, P, TR_SPLIT_W));
    TRY(elem(S->Wdd, S->TTdd, S->W3dd, S->eo_tri + t0, ns, S->maxbits, S->slot_ex, S->vptr,
             S->batch));
    if (prep) TRY(run(pZ.v[b], S->arrs, P, TR_SPLIT_OMEGA));
    TRY(run(pQ.v[b], aq, P, TR_SPLIT_OMEGA));
    TRY(run(pAB.v[b], jr, PR, TR_SPLIT_W));
    trace_begin(c, TR_SPLIT_ELEM, st);
    TRY(launch_left_outer_dd(Wj, tri_all + 3 * t0, bj, ns, nslot, l1dd, ltdd, ovdd, fdd, no, nv,
                             st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    *L += 1;
    // L3 of the batch: one exponent for all its slots (the grouped G jobs)
    trace_begin(c, TR_SPLIT_ELEM, st);
    CU(cudaMemsetAsync(maxj, 0, sizeof(unsigned int) * nslot, st));
    TRY(launch_tau_contravariant_dd(Wj, TTj, W3j, TTj, S->evdd, eoj_all + (size_t)b * nslot, 0.f,
                                    0.f, nv, nslot, maxj, st));
    TRY(launch_common_exponent(maxj, exj, nslot, bj, ns, st));
    TRY(launch_slice_tt(TTj, vptrj, nv, vp, s, exj, nslot, nslot, st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    *L += 3;
    TRY(run(pO.v[b], jr, PR, TR_SPLIT_OMEGA));
  }
  int hs = 0;
  CU(cudaMemcpyAsync(&hs, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (hs != 0) {
    cudaMemsetAsync(S->status, 0, sizeof(int), st);
    return hs == 2 ? CC3_FAIL(CC3_ERR_ARG, "a left-Jacobian plan addressed outside a slice array")
                   : CC3_FAIL(CC3_ERR_TIMEOUT, "split engine wait gave up");
  }
  if (prep) jac_set_prep(c, CC3_SPLIT_BF16);
  // The Cholesky product of sigma1, N[J][(c,k)] = sum_bd L^J_bd G[b][d][c][k]
  // (M = naux, N = nv no, K = nv^2), on the tensor cores: the slices of L^J_bd
  // once, those of each vector's G (its own exponent) per vector.
  const int naux = c->naux, n = no + nv;
  const long long nvo = (long long)nv * no, Kc = (long long)nv * vp;
  SArrTable ac = S->arrs;
  int Ech = 0;
  __nv_bfloat16 *gsl = nullptr;
  {
    __nv_bfloat16 *lch = nullptr;
    unsigned long long *mx = nullptr;
    TRY(B.get(&mx, 1));
    CU(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    TRY(launch_maxabs(c->chol, (long long)naux * n * n, mx, st));
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, mx, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double x;
    std::memcpy(&x, &hb, 8);
    Ech = exponent_of(x);
    const Gather g = {(long long)no * n + no, 0, 0, (long long)n * n, n, 1, 1, naux, vp,
                      nv, nv, 0};
    TRY(sliced(&lch, c->chol, naux, (int)Kc, Ech, g, naux));
    const size_t ng_sl = arr_elems(Kc, nvo, 1, s);
    TRY(B.get(&gsl, ng_sl));
    CU(cudaMemsetAsync(gsl, 0, ng_sl * sizeof(__nv_bfloat16), st));  // padding rows
    ac.a[ML_CHA] = make_arr(lch, Kc, naux, 1, s);
    ac.a[ML_GB] = make_arr(gsl, Kc, nvo, 1, s);
  }
  const int kspl = std::max(1, (int)((Kc / S_BK + S->ks_target - 1) / std::max(16, S->ks_target)));
  // sigma1 (FP64, from Q, G, H, N, Lt2 and Z~) and the pair-symmetric sigma2
  PtrTable pt;
  jac_fill_ptrs(c, &pt);
  pt.p[B_MJ] = N;
  VPtrTable PC = P;
  PC.p[B_MJ] = N;
  for (int v = 0; v < nvec; ++v) {
    double *Gv = G + v * ng;
    TRY(launch_zero(N, (size_t)naux * nvo, st));
    unsigned long long *mx = nullptr;
    TRY(B.get(&mx, 1));
    CU(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    TRY(launch_maxabs(Gv, (long long)ng, mx, st));
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, mx, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double x;
    std::memcpy(&x, &hb, 8);
    if (x > 0.0) {
      const int EG = exponent_of(x);
      const Gather g = {0, 0, 0, 1, (long long)nv * nvo, nvo, 1, (int)nvo, vp, nv, nv, 0};
      trace_begin(c, TR_SPLIT_ELEM, st);
      TRY(launch_slice_gather(Gv, gsl, s, EG, g, nvo, (int)Kc, (int)nvo, st));
      trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
      *L += 1;
      SPlan pc;
      const int jb = new_sjob(pc, naux, (int)nvo, ntile_for((int)nvo), 1, kspl, SEPI_F64_ATOMIC,
                              Ech + EG - 14, ex, s);
      pc.jobs[jb].C = outd(B_MJ, 0, nvo, 1);
      pc.jobs[jb].Ct = pc.jobs[jb].C;
      add_sterm(pc, jb, opd(ML_CHA, 0), opd(ML_GB, 0), (int)Kc, 0, ex, s);
      SDevPlan d;
      TRY(s_upload_plan(pc, &d, st));
      const int rc = run(d, ac, PC, TR_SPLIT_OMEGA);
      CU(cudaStreamSynchronize(st));  // the plan's tables are freed next
      s_free_plan(&d);
      TRY(rc);
    }
    pt.p[B_LT] = lt + v * nt2;
    pt.p[B_Q] = Q + v * n1;
    pt.p[B_G] = Gv;
    pt.p[B_H] = H + v * nh;
    pt.p[B_S1] = s1d + v * n1;
    TRY(launch_zero(s1d + v * n1, n1, st));
    TRY(left_finish(c, pt, s2raw + v * nt2, s2d + v * nt2, st, true));
  }
  {
    int hs2 = 0;
    CU(cudaMemcpyAsync(&hs2, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hs2 != 0) {
      cudaMemsetAsync(S->status, 0, sizeof(int), st);
      return hs2 == 2 ? CC3_FAIL(CC3_ERR_ARG, "a left-Jacobian plan addressed outside a slice array")
                      : CC3_FAIL(CC3_ERR_TIMEOUT, "split engine wait gave up");
    }
  }
  CU(cudaStreamSynchronize(st));
  c->counters.executed_flop += ex + ex_tau;
  c->counters.slices = s;
  return CC3_OK;
}

// ---- densities (Algorithm 3) on the tensor cores -----------------------------------
namespace {

// Y and D_vv jobs of one triple in slot u (L~ in the L3 layouts, tau in MD_TAU*):
//   Y[l][r][p][c] += sum_ab L~[a][b][c] t[l][q][a][b]   rows c of layout m2, K = (zb, u, zz)
//   Dvv[c][d]     += sum_ab L~[a][b][c] tau[a][b][d]    rows c of L~'s and d of tau's layout m2
void plan_density_split(SPlan &py, SPlan &pv, SplitState *S, int no, int nv, const int ijk[3],
                        int u, double &ex) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const int s = S->s, vp = S->vp;
  int seen[6][3], nseen = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int w = 0; w < 6; ++w) {
    const int *m = PERM6[w];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int x = 0; x < nseen; ++x)
      if (seen[x][0] == p && seen[x][1] == q && seen[x][2] == r) dup = true;
    if (dup) continue;
    seen[nseen][0] = p;
    seen[nseen][1] = q;
    seen[nseen][2] = r;
    ++nseen;
    const int Lz = m[2];
    const bool yz = (m[0] == (Lz + 1) % 3);  // K = (a, b) or (b, a)
    int jb = new_sjob(py, nv, no, ntile_for(no), 1, S->ks4, SEPI_F64_ATOMIC, S->Et - 14, ex, s);
    SJob &J = py.jobs[jb];
    J.expo_slot = u;
    J.C = outd(B_DY, ((long long)r * no + p) * nv, 1, (long long)no * no * nv);
    J.Ct = J.C;
    add_sterm(py, jb, opd(MA_V0 + Lz, u), opd(yz ? MD_T2YA : MD_T2YB, q), nv * vp, 0, ex, s);
    jb = new_sjob(pv, nv, nv, ntile_for(nv), 1, S->ks4, SEPI_F64_ATOMIC, -14, ex, s);
    SJob &K = pv.jobs[jb];
    K.expo_slot = u;  // in the array of summed exponents of L~ and tau
    K.C = outd(B_DVV, 0, nv, 1);
    K.Ct = K.C;
    add_sterm(pv, jb, opd(MA_V0 + Lz, u), opd(MD_TAU0 + Lz, u), nv * vp, 0, ex, s);
  }
}

}  // namespace

// Algorithm 3 on the tensor cores.  The occupied loop runs over the triples
// i >= j >= k and also i = j = k (tau there enters Doo): per batch tau3 (the
// residual's W build; the element-wise step also writes tau itself), the
// slices of tau, the Q jobs of the ov block, the L3 of the left state (as in
// the left transformation, one slice exponent for the batch), and the Y and
// D_vv jobs.  tau and L~3 of every triple stay resident (double-float), and
// Doo follows from them pair by pair (density_doo_resident) instead of the
// virtual loop; the calls that do not fit in memory return CC3_ERR_OOM.
int split_density(cc3_ctx *c, double w, const double *L1d, const double *L2d, double *Doo,
                  double *Dov, double *Dvv, cudaStream_t st) {
  SplitState *S = nullptr;
  TRY(split_ready(c, &S, st));
  const int no = c->no, nv = c->nv, s = S->s, vp = S->vp, op = S->op;
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv, oo = (long long)no * no;
  const long long onv = (long long)no * nv;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv;
  // the triples with i = j = k appended to the context's full list
  std::vector<int> ext(c->tri_host.begin(), c->tri_host.begin() + 3 * c->ntri);
  for (int i = 0; i < no; ++i) {
    ext.push_back(i);
    ext.push_back(i);
    ext.push_back(i);
  }
  const int next = (int)ext.size() / 3;
  JacBufs B;
  float2 *tau_all = nullptr, *lt_all = nullptr;
  {
    const size_t need = 2 * (size_t)next * (size_t)nv3 * sizeof(float2);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if (need > free_b / 2)
      return CC3_FAIL(CC3_ERR_OOM, "split densities: tau and L3 of every triple do not fit");
  }
  TRY(B.get(&tau_all, (size_t)next * nv3));
  TRY(B.get(&lt_all, (size_t)next * nv3));
  double *lt = nullptr, *Y = nullptr;
  float2 *l1dd = nullptr, *ltdd = nullptr, *ovdd = nullptr, *fdd = nullptr, *eo_ext = nullptr;
  int *tri_ext = nullptr;
  TRY(B.get(&lt, nt2));
  TRY(B.get(&Y, (size_t)(oo * no * nv)));
  TRY(B.get(&l1dd, n1));
  TRY(B.get(&ltdd, nt2));
  TRY(B.get(&ovdd, (size_t)(oo * nv2)));
  TRY(B.get(&fdd, n1));
  TRY(B.get(&eo_ext, (size_t)next));
  TRY(B.get(&tri_ext, 3 * (size_t)next));
  CU(cudaMemcpyAsync(tri_ext, ext.data(), sizeof(int) * ext.size(), cudaMemcpyHostToDevice, st));
  {
    std::vector<float2> h(next);
    for (int t = 0; t < next; ++t) {
      const dd::df e = dd::from_double_host(c->eo_h[ext[3 * t]] + c->eo_h[ext[3 * t + 1]] +
                                            c->eo_h[ext[3 * t + 2]]);
      h[t] = make_float2(e.hi, e.lo);
    }
    CU(cudaMemcpyAsync(eo_ext, h.data(), sizeof(float2) * next, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
  }
  TRY(launch_zero(Doo, (size_t)oo, st));
  TRY(launch_zero(Dov, n1, st));
  TRY(launch_zero(Dvv, (size_t)nv2, st));
  TRY(launch_zero(Y, (size_t)(oo * no * nv), st));
  TRY(launch_back_transform(L2d, lt, no, nv, st));
  TRY(launch_to_dd(L1d, l1dd, (long long)n1, st));
  TRY(launch_to_dd(lt, ltdd, (long long)nt2, st));
  TRY(launch_to_dd(c->ovov, ovdd, oo * nv2, st));
  TRY(launch_to_dd(c->F_ov, fdd, (long long)n1, st));
  int ELt = 0;
  {
    unsigned long long *mx = nullptr;
    TRY(B.get(&mx, 1));
    CU(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
    TRY(launch_maxabs(lt, (long long)nt2, mx, st));
    unsigned long long hb = 0;
    CU(cudaMemcpyAsync(&hb, mx, sizeof(hb), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double x;
    std::memcpy(&x, &hb, 8);
    ELt = x > 0.0 ? exponent_of(x) : 0;
  }
  auto sliced = [&](__nv_bfloat16 **dst, const double *src, long long rows, int Kp, int E,
                    const Gather &g, int rps) -> int {
    const size_t n = arr_elems(Kp, rps, rows / rps, s);
    TRY(B.get(dst, n));
    CU(cudaMemsetAsync(*dst, 0, n * sizeof(__nv_bfloat16), st));
    return launch_slice_gather(src, *dst, s, E, g, rows, Kp, rps, st);
  };
  SArrTable jr = S->arrs, aq = S->arrs;
  {
    __nv_bfloat16 *tya = nullptr, *tyb = nullptr, *lqa = nullptr, *lqb = nullptr;
    Gather g;
    // t2 for Y: [q][l][(u,w)] = t[l][q][u][w] (YA) or t[l][q][w][u] (YB)
    g = {0, 0, nv2, (long long)no * nv2, nv, 1, no, no, nv, nv, nv, 1};
    TRY(sliced(&tya, c->t2, oo, nv * vp, S->Et, g, no));
    g = {0, 0, nv2, (long long)no * nv2, 1, nv, no, no, nv, nv, nv, 1};
    TRY(sliced(&tyb, c->t2, oo, nv * vp, S->Et, g, no));
    // Lt2 for Q (one vector): rows 0 of slab (p,q)
    g = {0, nv2, 0, 0, nv, 1, 1, 1, nv, nv, nv, 1};
    TRY(sliced(&lqa, lt, oo, nv * vp, ELt, g, 1));
    g = {0, nv2, 0, 0, 1, nv, 1, 1, nv, nv, nv, 1};
    TRY(sliced(&lqb, lt, oo, nv * vp, ELt, g, 1));
    jr.a[MD_T2YA] = make_arr(tya, (long long)nv * vp, no, no, s);
    jr.a[MD_T2YB] = make_arr(tyb, (long long)nv * vp, no, no, s);
    aq.a[ML_LQA] = make_arr(lqa, (long long)nv * vp, 1, oo, s);
    aq.a[ML_LQB] = make_arr(lqb, (long long)nv * vp, 1, oo, s);
  }
  // Lt2 in the t2 roles of the W build
  {
    struct Kind {
      int map;
      long long K, rps, slabs;
    };
    const Kind kinds[3] = {{MJ_R2S, vp, nv, oo}, {MJ_R2C, op, nv, onv}, {MJ_R2R, op, nv, onv}};
    const Gather gs[3] = {{0, (long long)no * nv2, nv2, nv, 0, 1, no, nv, vp, nv, 1, 0},
                          {0, (long long)no * nv2, 1, nv, 0, nv2, nv, nv, op, no, 1, 0},
                          {0, (long long)no * nv2, nv, 1, 0, nv2, nv, nv, op, no, 1, 0}};
    for (int i = 0; i < 3; ++i) {
      __nv_bfloat16 *a = nullptr;
      TRY(sliced(&a, lt, kinds[i].slabs * kinds[i].rps, (int)kinds[i].K, ELt, gs[i],
                 (int)kinds[i].rps));
      jr.a[kinds[i].map] = make_arr(a, kinds[i].K, kinds[i].rps, kinds[i].slabs, s);
    }
  }
  // per batch: L3 slots (the residual's batch size), the slices of L~ and of tau
  const int bj = S->batch;
  float2 *Wj = nullptr, *TTj = nullptr, *W3j = nullptr, *eol = nullptr;
  __nv_bfloat16 *Vj[3] = {nullptr, nullptr, nullptr}, *Vt[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16 **vptrj = nullptr, **vptrt = nullptr;
  unsigned int *maxj = nullptr, *maxt = nullptr;
  int *exj = nullptr, *ext_ = nullptr, *exs = nullptr;
  TRY(B.get(&Wj, (size_t)bj * nv3));
  TRY(B.get(&TTj, (size_t)bj * nv3));
  TRY(B.get(&W3j, (size_t)bj * nv3));
  TRY(B.get(&eol, (size_t)next));
  TRY(B.get(&maxj, (size_t)bj));
  TRY(B.get(&maxt, (size_t)bj));
  TRY(B.get(&exj, (size_t)bj));
  TRY(B.get(&ext_, (size_t)bj));
  TRY(B.get(&exs, (size_t)bj));
  TRY(B.get(&vptrj, 3));
  TRY(B.get(&vptrt, 3));
  const long long nv8 = (nv + 7) / 8 * 8;
  for (int L = 0; L < 3; ++L) {
    const size_t n4 = arr_elems((long long)nv * vp, nv, bj, s);
    TRY(B.get(&Vj[L], n4));
    TRY(B.get(&Vt[L], n4));
    CU(cudaMemsetAsync(Vj[L], 0, n4 * sizeof(__nv_bfloat16), st));
    CU(cudaMemsetAsync(Vt[L], 0, n4 * sizeof(__nv_bfloat16), st));
    jr.a[MA_V0 + L] = make_arr(Vj[L], (long long)nv * vp, nv, bj, s);
    jr.a[MA_V0K + L] = make_arr(Vj[L], vp, (long long)nv * nv8, bj, s);
    jr.a[MD_TAU0 + L] = make_arr(Vt[L], (long long)nv * vp, nv, bj, s);
  }
  CU(cudaMemcpyAsync(vptrj, Vj, sizeof(Vj), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(vptrt, Vt, sizeof(Vt), cudaMemcpyHostToDevice, st));
  {
    std::vector<float2> h(next);
    for (int t = 0; t < next; ++t) {
      const dd::df e = dd::from_double_host(c->eo_h[ext[3 * t]] + c->eo_h[ext[3 * t + 1]] +
                                            c->eo_h[ext[3 * t + 2]] + w);
      h[t] = make_float2(e.hi, e.lo);
    }
    CU(cudaMemcpyAsync(eol, h.data(), sizeof(float2) * next, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
  }
  const int rows = (nv + 7) / 8 * 8;
  const int Ec = ELt + S->Eg;
  VPtrTable P;
  fill_vptrs(c, S, &P);
  P.p[B_Q] = Dov;
  VPtrTable PR = P;
  PR.p[B_WS_W] = Wj;
  PR.p[B_WS_TT] = TTj;
  PR.p[B_WS_W3] = W3j;
  PR.p[B_SLOTEXP] = exj;
  PR.p[B_DY] = Y;
  VPtrTable PV = PR;
  PV.p[B_SLOTEXP] = exs;
  PV.p[B_DVV] = Dvv;
  const int kd = S_DRAIN_STEPS;
  long long *Lc = &c->counters.launches;
  double ex = 0.0;
  auto run = [&](const SPlan &p, const SArrTable &a, const VPtrTable &pt, int cls) -> int {
    if (p.jobs.empty()) return CC3_OK;
    SDevPlan d;
    TRY(s_upload_plan(p, &d, st));
    trace_begin(c, cls, st);
    const int rc = s_launch_plan(d, a, pt, s, kd, S->status, st, Lc);
    trace_end(c, cls, st, d.flop, d.slice_flop);
    CU(cudaStreamSynchronize(st));  // the tables are freed next
    s_free_plan(&d);
    return rc;
  };
  for (int t0 = 0; t0 < next; t0 += bj) {
    const int t1 = std::min(next, t0 + bj), ns = t1 - t0;
    SPlan tb, qp, ab, py, pv;
    for (int t = t0; t < t1; ++t) {
      const int *ijk = &ext[3 * t];
      plan_w_split(tb, S, no, nv, ijk, t - t0, ex);
      plan_left_split(nullptr, &qp, nullptr, S, no, nv, ELt, 1, ijk, t - t0, 0, 0, ex);
      WMaps set1 = {MJ_R2S, MJ_R2S, MJ_R2C, MJ_R2C, MJ_R2R, MJ_R2R,
                    MA_XS,  MB_XS,  MA_YS,  MB_YS,  MA_OS,  MB_OS};
      const int u = t - t0;
      const int j1 = w_job(ab, nv, rows, S->Nab, 1, u, Ec - 14, ex, s);
      w_terms_1(ab, j1, set1, no, nv, rows, vp, op, ijk, ex, s);
      const int j2 = w_job(ab, nv, rows, S->Nab, 2, u, Ec - 14, ex, s);
      w_terms_2(ab, j2, set1, no, nv, rows, vp, op, ijk, ex, s);
      const int j3 = w_job(ab, nv, rows, S->Nab, 3, u, Ec - 14, ex, s);
      w_terms_3(ab, j3, set1, no, nv, rows, vp, op, ijk, ex, s);
      plan_density_split(py, pv, S, no, nv, ijk, u, ex);
    }
    // tau: W build, then tau (resident) and tau~ with its slices
    TRY(run(tb, S->arrs, P, TR_SPLIT_W));
    trace_begin(c, TR_SPLIT_ELEM, st);
    CU(cudaMemsetAsync(S->maxbits, 0, sizeof(unsigned int) * ns, st));
    TRY(launch_tau_contravariant_dd(S->Wdd, S->TTdd, S->W3dd, S->TTdd, S->evdd, eo_ext + t0, 0.f,
                                    0.f, nv, ns, S->maxbits, st, tau_all + (size_t)t0 * nv3));
    TRY(launch_slot_exponent(S->maxbits, S->slot_ex, ns, st));
    TRY(launch_slice_tt(S->TTdd, S->vptr, nv, vp, s, S->slot_ex, ns, S->batch, st));
    // the slices of tau itself, one exponent for the batch
    CU(cudaMemsetAsync(maxt, 0, sizeof(unsigned int) * bj, st));
    TRY(launch_slot_maxabs_dd(tau_all + (size_t)t0 * nv3, nv3, ns, maxt, st));
    TRY(launch_common_exponent(maxt, ext_, bj, bj, ns, st));
    TRY(launch_slice_tt(tau_all + (size_t)t0 * nv3, vptrt, nv, vp, s, ext_, ns, bj, st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    *Lc += 7;
    TRY(run(qp, aq, P, TR_SPLIT_OMEGA));
    // L3 of the left state: W-build bracket, outer products, (w - eps), L~ (one
    // exponent for the batch) with its slices, kept resident
    TRY(run(ab, jr, PR, TR_SPLIT_W));
    trace_begin(c, TR_SPLIT_ELEM, st);
    TRY(launch_left_outer_dd(Wj, tri_ext + 3 * t0, bj, ns, ns, l1dd, ltdd, ovdd, fdd, no, nv, st));
    CU(cudaMemsetAsync(maxj, 0, sizeof(unsigned int) * bj, st));
    TRY(launch_tau_contravariant_dd(Wj, TTj, W3j, TTj, S->evdd, eol + t0, 0.f, 0.f, nv, ns, maxj,
                                    st));
    TRY(launch_common_exponent(maxj, exj, bj, bj, ns, st));
    TRY(launch_slice_tt(TTj, vptrj, nv, vp, s, exj, ns, bj, st));
    CU(cudaMemcpyAsync(lt_all + (size_t)t0 * nv3, TTj, sizeof(float2) * (size_t)ns * nv3,
                       cudaMemcpyDeviceToDevice, st));
    TRY(launch_add_int(exj, ext_, exs, bj, st));
    trace_end(c, TR_SPLIT_ELEM, st, 0.0, 0.0);
    *Lc += 6;
    TRY(run(py, jr, PR, TR_SPLIT_OMEGA));
    TRY(run(pv, jr, PV, TR_SPLIT_OMEGA));
  }
  int hs = 0;
  CU(cudaMemcpyAsync(&hs, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (hs != 0) {
    cudaMemsetAsync(S->status, 0, sizeof(int), st);
    return hs == 2 ? CC3_FAIL(CC3_ERR_ARG, "a density plan addressed outside a slice array")
                   : CC3_FAIL(CC3_ERR_TIMEOUT, "split engine wait gave up");
  }
  // the end of the occupied loop and Doo, in FP64
  PtrTable pt;
  jac_fill_ptrs(c, &pt);
  pt.p[B_DY] = Y;
  pt.p[B_DOV] = Dov;
  TRY(density_tail(c, pt, Dvv, st));
  TRY(density_doo_resident(c, tau_all, lt_all, ext, Doo, st));
  c->counters.executed_flop += ex;
  c->counters.slices = s;
  return CC3_OK;
}

// Device bytes of one split Jacobian call beyond the residual's state: the
// Algorithm 2 layouts of ovov, FP64 dressed blocks and the slices of R2 and
// g^ of every vector.
size_t split_jacobian_footprint(int no, int nv, int s, int nvec) {
  const int vp = rup(nv, 16), op = rup(no, 16);
  auto sl = [&](long long rows, long long Kp, long long rps) {
    return arr_elems(Kp, rps, rows / rps, s) * sizeof(__nv_bfloat16);
  };
  size_t b = sl((long long)no * no * nv, vp, nv) + 2 * sl((long long)no * no, (long long)nv * vp, no);
  size_t per = sl((long long)no * no * nv, vp, nv) + 2 * sl((long long)no * nv * nv, op, nv) +
               2 * sl((long long)no * nv * nv, vp, nv) + sl((long long)no * no * nv, op, nv);
  b += (size_t)nvec * per + sl((long long)no * nvec, vp, nvec);
  // the R3 slots of all vectors (the same arithmetic as split_jacobian)
  const long long nv2 = (long long)nv * nv;
  const double per_slot = (double)nv2 * nv * 24.0 + 3.0 * s * nv2 * vp * 2.0;
  const int batch = (int)std::max(1.0, std::min(16.0, 6.0e9 / per_slot));
  const int bj = std::max(1, std::min(batch, (int)(12.0e9 / (per_slot * nvec))));
  b += (size_t)(nvec * bj) * (size_t)(3 * nv2 * nv * sizeof(float2) + 16) +
       3 * arr_elems((long long)nv * vp, nv, (long long)nvec * bj, s) * sizeof(__nv_bfloat16);
  return b + 65536;
}

// ---- diagnostic: one plain GEMM C[m][n] = sum_k A[m][k] B[n][k] ------------------
int debug_split_gemm(int M, int N, int K, const double *A, const double *B, double *C, int s,
                     cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1 || s < 3 || s > S_MAX_SLICES) return CC3_ERR_ARG;
  const int Kp = rup(K, 16);
  const int Nt = ntile_for(N);
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  __nv_bfloat16 *sA = nullptr, *sB = nullptr;
  unsigned long long *mx = nullptr;
  int *status = nullptr;
  int rc = CC3_OK;
  SPlan P;
  SDevPlan D;
  SArrTable arrs;
  VPtrTable ptr;
  double ex = 0.0;
  unsigned long long h[2];
  double ma, mb;
  Gather gA, gB;
  std::memset(&arrs, 0, sizeof(arrs));
  std::memset(&ptr, 0, sizeof(ptr));
#define CK(x)                    \
  do {                           \
    if ((rc = (x)) != CC3_OK) goto done; \
  } while (0)
#define CKC(x)                                   \
  do {                                           \
    if ((x) != cudaSuccess) { rc = CC3_FAIL(CC3_ERR_CUDA, "debug gemm cuda call"); goto done; } \
  } while (0)
  CK(alloc(&dA, (size_t)M * K));
  CK(alloc(&dB, (size_t)N * K));
  CK(alloc(&dC, (size_t)M * N));
  CK(alloc(&sA, arr_elems(Kp, M, 1, s)));
  CK(alloc(&sB, arr_elems(Kp, N, 1, s)));
  CKC(cudaMemsetAsync(sA, 0, arr_elems(Kp, M, 1, s) * 2, st));
  CKC(cudaMemsetAsync(sB, 0, arr_elems(Kp, N, 1, s) * 2, st));
  CK(alloc(&mx, 2));
  CK(alloc(&status, 1));
  CKC(cudaMemcpyAsync(dA, A, sizeof(double) * M * K, cudaMemcpyHostToDevice, st));
  CKC(cudaMemcpyAsync(dB, B, sizeof(double) * N * K, cudaMemcpyHostToDevice, st));
  CKC(cudaMemsetAsync(dC, 0, sizeof(double) * M * N, st));
  CKC(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), st));
  CKC(cudaMemsetAsync(status, 0, sizeof(int), st));
  CK(launch_maxabs(dA, (long long)M * K, mx, st));
  CK(launch_maxabs(dB, (long long)N * K, mx + 1, st));
  CKC(cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, st));
  CKC(cudaStreamSynchronize(st));
  std::memcpy(&ma, &h[0], 8);
  std::memcpy(&mb, &h[1], 8);
  {
    const int eA = exponent_of(ma), eB = exponent_of(mb);
    gA = {0, 0, 0, K, 0, 1, 1, 1 << 30, Kp, K, 1};
    gA.n1 = 1;
    gA.n0 = 1 << 30;
    gB = gA;
    CK(launch_slice_gather(dA, sA, s, eA, gA, M, Kp, M, st));
    CK(launch_slice_gather(dB, sB, s, eB, gB, N, Kp, N, st));
    arrs.a[0] = make_arr(sA, Kp, M, 1, s);
    arrs.a[1] = make_arr(sB, Kp, N, 1, s);
    int jb = new_sjob(P, M, N, Nt, 1, 1, SEPI_F64_ATOMIC, eA + eB - 14, ex, s);
    P.jobs[jb].C = outd(0, 0, N, 1);
    P.jobs[jb].Ct = P.jobs[jb].C;
    add_sterm(P, jb, opd(0, 0), opd(1, 0), Kp, 0, ex, s);
    CK(s_upload_plan(P, &D, st));
    ptr.p[0] = dC;
    CK(s_launch_plan(D, arrs, ptr, s, S_DRAIN_STEPS, status, st, nullptr));
    int hs = 0;
    CKC(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(C, dC, sizeof(double) * M * N, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (hs) rc = CC3_ERR_TIMEOUT;
  }
done:
  s_free_plan(&D);
  void *bufs[] = {dA, dB, dC, sA, sB, mx, status};
  for (void *p : bufs)
    if (p) cudaFree(p);
  cudaGetLastError();
  return rc;
#undef CK
#undef CKC
}

}  // namespace cc3

extern "C" int cc3_debug_split_gemm(int M, int N, int K, const double *A, const double *B,
                                    double *C, int slices) {
  return cc3::debug_split_gemm(M, N, K, A, B, C, slices, nullptr);
}
