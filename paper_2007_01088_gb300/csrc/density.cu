// Triples contributions to the one-electron density of a left state
// (Algorithm 3), FP64 path: D^{m,0}_{pq} = <m|E_pq|CC> for a left state
// (L1, L2) at frequency w, or D^{0,0} with the ground-state multipliers at
// w = 0.  The vo block has no triples term.
//
// Occupied loop, batches of the triples i >= j >= k, every distinct
// permutation (p,q,r) of a triple (views with the virtual slots permuted
// alike):
//   tau (covariant, [c][a][b] per slot) and tau~ from the residual's W build;
//   L3 = P X / (w - eps) and L~ from the left transformation's builder (X from
//   L1 and Lt2, the back-transformed L2);
//   Y[l][r][p][c] += sum_ab L~_pqr[a][b][c] t[l][q][a][b]
//   Dvv[c][d]     += sum_ab L~_pqr[a][b][c] tau_pqr[a][b][d]     (halved at the end)
//   Dov[r][c]     += sum_ab Lt2[p][q][a][b] tau~_pqr[a][b][c]
// then Dov[l][d] -= sum_{k,i,c} Y[l][k][i][c] t[k][i][c][d].
//
// Virtual loop (the loop a >= b >= c of Algorithm 3), by slabs of the largest
// virtual index A, several small slabs per launch: the brackets
//   B^{xyz}_{pqr} = sum_d t^{xd}_{pq} (yd|zr) - sum_l t^{xy}_{pl} (lq|zr)
// of every ordered (x,y,z) whose largest index is A, in three groups (x = A,
// y = A, z = A; each [first free][second free][p][q][r]), and the same
// brackets of Lt2 (the L2 contractions of the L3 numerator), are engine
// contractions over all (p,q,r): the d-sums stored, then the l-sums added.
// One kernel then takes each virtual triple (A, b, c), forms tau^{Abc}_{ijk}
// and L3^{Abc}_{ijk} for all (i,j,k) in shared memory (six bracket terms of
// P plus the outer products L^x_p (qy|rz) + Lt2^{xy}_{pq} F_rz), turns L3
// into L~ in place by the occupied permutations
//   L~^{abc}_{ijk} = 4 L_{ijk} - 2 L_{ikj} - 2 L_{kji} - 2 L_{jik} + L_{kij} + L_{jki}
// (every term at virtual order (a,b,c), by the six-fold symmetry), and adds
//   Doo[l][k] -= (n / 6) sum_s sum_{other two slots} L~[.. k in slot s ..] tau[.. l in slot s ..]
// which is Algorithm 3's sum over the n distinct orderings of (A, b, c),
// grouped by the slot s that the third virtual index comes from.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
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

constexpr int DV_THREADS = 256;
constexpr int DV_MAX_NO = 24;  // tau and L3 of one virtual triple in shared memory

__global__ void scale_kernel(double *x, long long n, double a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] *= a;
}

// Doo contributions of the virtual triples of slabs [A0, A1) (see the header).
// Bt, Bx: the tau and L3 brackets of the group, slab A at 3 G(A) no^3 (G(A) =
// sum over the group's slabs below A of (A'+1)^2), its three groups (x = A,
// y = A, z = A) (A+1)^2 no^3 apart.
__global__ void __launch_bounds__(DV_THREADS)
density_virtual_kernel(const double *__restrict__ Bt, const double *__restrict__ Bx, int A0,
                       int A1, long long ntrip, const double *__restrict__ lt,
                       const double *__restrict__ L1, const double *__restrict__ ovov,
                       const double *__restrict__ F, const double *__restrict__ eo,
                       const double *__restrict__ ev, double w, int no, int nv,
                       double *__restrict__ Doo) {
  // the six slot maps (as PERM6) and kComp[u][m] = the index of the map
  // t -> kP6[u][kP6[m][t]]; compile-time tables, so that the unrolled loops
  // index registers
  constexpr int kP6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0}, {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  constexpr int kComp[6][6] = {{0, 1, 2, 3, 4, 5}, {1, 0, 5, 4, 3, 2}, {2, 4, 0, 5, 1, 3},
                               {3, 5, 4, 0, 2, 1}, {4, 2, 3, 1, 5, 0}, {5, 3, 1, 2, 0, 4}};
  extern __shared__ double dsm[];
  const int no2 = no * no, no3 = no2 * no;
  double *tau = dsm, *lc = dsm + no3;
  double acc[(DV_MAX_NO * DV_MAX_NO + DV_THREADS - 1) / DV_THREADS];
#pragma unroll
  for (int u = 0; u < (int)(sizeof(acc) / sizeof(acc[0])); ++u) acc[u] = 0.0;
  const long long g0 = (long long)A0 * (A0 + 1) * (2 * A0 + 1) / 6;
  for (long long g = blockIdx.x; g < ntrip; g += gridDim.x) {
    // (A, b, c): slab by slab, pairs c <= b <= A in order, (A, A, A) left out
    long long r = g;
    int A = A0;
    for (; A < A1; ++A) {
      const long long cnt = (long long)(A + 1) * (A + 2) / 2 - 1;
      if (r < cnt) break;
      r -= cnt;
    }
    int b = (int)((sqrt(8.0 * (double)r + 1.0) - 1.0) * 0.5);
    while ((long long)(b + 1) * (b + 2) / 2 <= r) ++b;
    while ((long long)b * (b + 1) / 2 > r) --b;
    const int c = (int)(r - (long long)b * (b + 1) / 2);
    const int v[3] = {A, b, c};
    const double wv = (A != b && b != c) ? 1.0 : 0.5;  // distinct orderings / 6
    const long long base = 3 * ((long long)A * (A + 1) * (2 * A + 1) / 6 - g0) * no3;
    const long long A1p = A + 1, sz = A1p * A1p * no3;
    const double ev3 = ev[A] + ev[b] + ev[c];
    __syncthreads();  // the previous triple's reads of tau and lc are done
    for (int e = threadIdx.x; e < no3; e += blockDim.x) {
      const int o[3] = {e / no2, (e / no) % no, e % no};
      double wt = 0.0, wx = 0.0;
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const int x = v[kP6[u][0]], y = v[kP6[u][1]], z = v[kP6[u][2]];
        const int p = o[kP6[u][0]], q = o[kP6[u][1]], rr = o[kP6[u][2]];
        long long reg;
        if (x == A)
          reg = base + ((long long)y * A1p + z) * no3;
        else if (y == A)
          reg = base + sz + ((long long)x * A1p + z) * no3;
        else
          reg = base + 2 * sz + ((long long)x * A1p + y) * no3;
        const long long idx = reg + ((long long)p * no + q) * no + rr;
        wt += Bt[idx];
        wx += Bx[idx] + L1[(long long)p * nv + x] * ovov[(((long long)q * nv + y) * no + rr) * nv + z] +
              lt[(((long long)p * no + q) * nv + x) * nv + y] * F[(long long)rr * nv + z];
      }
      const double den = ev3 - eo[o[0]] - eo[o[1]] - eo[o[2]];
      tau[e] = wt / (0.0 - den);
      lc[e] = wx / (w - den);
    }
    __syncthreads();
    // L~ in place, one orbit {i >= j >= k} of occupied permutations per thread
    for (int e = threadIdx.x; e < no3; e += blockDim.x) {
      const int o[3] = {e / no2, (e / no) % no, e % no};
      if (!(o[0] >= o[1] && o[1] >= o[2])) continue;
      int pos[6];
      double L[6];
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        pos[u] = (o[kP6[u][0]] * no + o[kP6[u][1]]) * no + o[kP6[u][2]];
        L[u] = lc[pos[u]];
      }
      double T[6];
#pragma unroll
      for (int u = 0; u < 6; ++u)
        T[u] = 4.0 * L[kComp[u][0]] - 2.0 * L[kComp[u][3]] - 2.0 * L[kComp[u][2]] -
               2.0 * L[kComp[u][1]] + L[kComp[u][5]] + L[kComp[u][4]];
#pragma unroll
      for (int u = 0; u < 6; ++u) lc[pos[u]] = T[u];
    }
    __syncthreads();
    int slot = 0;
    for (int pi = threadIdx.x; pi < no2; pi += blockDim.x, ++slot) {
      const int l = pi / no, k = pi % no;
      double s = 0.0;
      for (int x = 0; x < no2; ++x) s += lc[k * no2 + x] * tau[l * no2 + x];  // slot 0
      for (int i = 0; i < no; ++i)                                            // slot 1
        for (int kk = 0; kk < no; ++kk) s += lc[(i * no + k) * no + kk] * tau[(i * no + l) * no + kk];
      for (int x = 0; x < no2; ++x) s += lc[x * no + k] * tau[x * no + l];    // slot 2
      acc[slot] -= wv * s;
    }
  }
  int slot = 0;
  for (int pi = threadIdx.x; pi < no2; pi += blockDim.x, ++slot)
    if (acc[slot] != 0.0) atomicAdd(&Doo[pi], acc[slot]);
}

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
      return CC3_FAIL(CC3_ERR_OOM, "density workspace");
    }
    p.push_back(*out);
    return CC3_OK;
  }
};

int grid_for(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, 8192LL)); }

// Y and Dvv jobs of one triple in slot `slot` (L~ in B_WS_TTR as [a][b][c],
// tau in B_WS_W as [c][a][b])
void plan_density_occ(Plan &py, Plan &pv, int no, int nv, const int ijk[3], int slot) {
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long stL[3] = {nv2, nv, 1}, stT[3] = {nv, 1, nv2};
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  int seen[6][3], ns = 0;
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
    const Opnd Lv = with_k2(op(B_WS_TTR, slot * nv3, stL[m[2]], stL[m[1]]), nv, stL[m[0]]);
    // Y[l][r][p][c]: rows c, cols l, K = (a, b)
    int jb = new_job(py, 1, nv, no, no, 1, 1, EPI_ATOMIC);
    add_term(py, jb, Lv, op(B_T2, (long long)q * nv2, (long long)no * nv2, 1), (int)nv2);
    OutD o = out(B_DY, ((long long)r * no + p) * nv, 1, (long long)no * no * nv);
    py.jobs[jb].C = o;
    py.jobs[jb].Ct = o;
    // Dvv[c][d]: rows c, cols d, K = (a, b)
    jb = new_job(pv, 0, nv, nv, nv, 1, 1, EPI_ATOMIC);
    add_term(pv, jb, Lv, with_k2(op(B_WS_W, slot * nv3, stT[m[2]], stT[m[1]]), nv, stT[m[0]]),
             (int)nv2);
    o = out(B_DVV, 0, nv, 1);
    pv.jobs[jb].C = o;
    pv.jobs[jb].Ct = o;
  }
}

// The brackets of slab A (d-sums into p1, stored; l-sums into p2, added) for
// tau (t2 -> buffer B_VBT) and for L3 (Lt2 -> B_VBX), at `base` in those
// buffers.
void plan_virtual_brackets(Plan &p1, Plan &p2, int no, int nv, int A, long long base) {
  const long long no2 = (long long)no * no, no3 = no2 * no, A1p = A + 1;
  const long long nv2 = (long long)nv * nv, nvo = (long long)nv * no, nv2o = nv2 * no;
  const long long sz = A1p * A1p * no3;
  const int N1 = (int)(A1p * no);
  const int bufs[2] = {B_VBT, B_VBX}, amps[2] = {B_T2, B_LT};
  for (int h = 0; h < 2; ++h) {
    const int ob = bufs[h], tb = amps[h];
    // d-sums: rows (p, q), cols (second free index, r), batch = first free index
    auto store = [&](long long off) {
      OutD o = out(ob, base + off, no, 1, A1p * no3);
      o.n_in = no;
      o.sn1 = no3;
      return o;
    };
    int jb = new_job(p1, 0, (int)no2, N1, N1, (int)A1p, 1, EPI_STORE);  // x = A: batch y
    add_term(p1, jb, op(tb, (long long)A * nv, nv2, 1, 0), op(B_VVVO, 0, 1, nvo, nv2o), nv);
    p1.jobs[jb].C = p1.jobs[jb].Ct = store(0);
    jb = new_job(p1, 0, (int)no2, N1, N1, (int)A1p, 1, EPI_STORE);  // y = A: batch x
    add_term(p1, jb, op(tb, 0, nv2, 1, nv), op(B_VVVO, (long long)A * nv2o, 1, nvo, 0), nv);
    p1.jobs[jb].C = p1.jobs[jb].Ct = store(sz);
    jb = new_job(p1, 0, (int)no2, N1, N1, (int)A1p, 1, EPI_STORE);  // z = A: batch x
    add_term(p1, jb, op(tb, 0, nv2, 1, nv),
             with_m2(op(B_VVVO, (long long)A * no, 1, nvo, 0), no, nv2o), nv);
    p1.jobs[jb].C = p1.jobs[jb].Ct = store(2 * sz);
    // l-sums, subtracted: rows (first or second free index, p), cols (q, r)
    auto add = [&](long long off, long long sm1, long long sb) {
      OutD o = out(ob, base + off, no2, 1, sb);
      o.m_in = no;
      o.sm1 = sm1;
      o.n_in = no;
      o.sn1 = no;
      return o;
    };
    const Opnd G = with_m2(op(B_OOVO, 0, 1, no * nvo, no), no, nvo);  // (lq|zr), batch z
    // x = A: rows (y, p), batch z
    jb = new_job(p2, 0, N1, (int)no2, (int)no2, (int)A1p, 1, EPI_ATOMIC);
    add_term(p2, jb, with_m2(op(tb, (long long)A * nv, no * nv2, nv2, 0, 1), no, 1), G, no);
    p2.jobs[jb].C = p2.jobs[jb].Ct = add(0, A1p * no3, no3);
    // y = A: rows (x, p), batch z
    jb = new_job(p2, 0, N1, (int)no2, (int)no2, (int)A1p, 1, EPI_ATOMIC);
    add_term(p2, jb, with_m2(op(tb, A, no * nv2, nv2, 0, 1), no, nv), G, no);
    p2.jobs[jb].C = p2.jobs[jb].Ct = add(sz, A1p * no3, no3);
    // z = A: rows (y, p), batch x, (lq|Ar)
    jb = new_job(p2, 0, N1, (int)no2, (int)no2, (int)A1p, 1, EPI_ATOMIC);
    add_term(p2, jb, with_m2(op(tb, 0, no * nv2, nv2, nv, 1), no, 1),
             with_m2(op(B_OOVO, (long long)A * no, 1, no * nvo, 0), no, nvo), no);
    p2.jobs[jb].C = p2.jobs[jb].Ct = add(2 * sz, no3, A1p * no3);
  }
}

int density_virtual(cc3_ctx *c, PtrTable pt, double w, const double *L1d, const double *ltd,
                    double *Doo, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const long long no3 = (long long)no * no * no, cap = (long long)nv * nv;
  Bufs B;
  double *Bt = nullptr, *Bx = nullptr;
  TRY(B.get(&Bt, (size_t)(3 * cap * no3)));
  TRY(B.get(&Bx, (size_t)(3 * cap * no3)));
  pt.p[B_VBT] = Bt;
  pt.p[B_VBX] = Bx;
  {
    static std::mutex mu;
    static bool set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && !set[dev]) {
      CU(cudaFuncSetAttribute(density_virtual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(2 * sizeof(double) * DV_MAX_NO * DV_MAX_NO * DV_MAX_NO)));
      set[dev] = true;
    }
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const size_t smem = 2 * sizeof(double) * (size_t)no3;
  for (int A0 = 0; A0 < nv;) {
    int A1 = A0;
    long long used = 0, ntrip = 0;
    while (A1 < nv && (A1 == A0 || used + (long long)(A1 + 1) * (A1 + 1) <= cap)) {
      used += (long long)(A1 + 1) * (A1 + 1);
      ntrip += (long long)(A1 + 1) * (A1 + 2) / 2 - 1;
      ++A1;
    }
    Plan p1, p2;
    long long base = 0;
    for (int A = A0; A < A1; ++A) {
      plan_virtual_brackets(p1, p2, no, nv, A, base);
      base += 3LL * (A + 1) * (A + 1) * no3;
    }
    TRY(jac_run_plan(c, p1, 0, pt, s));
    TRY(jac_run_plan(c, p2, 0, pt, s));
    if (ntrip > 0) {
      const int grid = (int)std::min<long long>(ntrip, 2LL * std::max(1, sms));
      trace_begin(c, TR_FP64_ELEM, s);
      density_virtual_kernel<<<grid, DV_THREADS, smem, s>>>(Bt, Bx, A0, A1, ntrip, ltd, L1d,
                                                            c->ovov, c->F_ov, c->eps_o,
                                                            c->eps_v, w, no, nv, Doo);
      CU(cudaGetLastError());
      trace_end(c, TR_FP64_ELEM, s, 0.0, 0.0);
      c->counters.launches++;
    }
    A0 = A1;
  }
  CU(cudaStreamSynchronize(s));  // the bracket buffers are freed next
  return CC3_OK;
}

int density_fp64(cc3_ctx *c, double w, const double *L1d, const double *L2d, double *Doo,
                 double *Dov, double *Dvv, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv, no3 = (long long)no * no * no;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv;
  Bufs B;
  double *lt = nullptr, *Y = nullptr, *wsW = nullptr, *wsT = nullptr;
  int *tri = nullptr;
  TRY(B.get(&lt, nt2));
  TRY(B.get(&Y, (size_t)(no3 * nv)));
  TRY(B.get(&wsW, (size_t)nv3 * c->batch));
  TRY(B.get(&wsT, (size_t)nv3 * c->batch));
  TRY(B.get(&tri, 3 * (size_t)c->batch));
  TRY(launch_zero(Doo, (size_t)no * no, s));
  TRY(launch_zero(Dov, n1, s));
  TRY(launch_zero(Dvv, (size_t)nv2, s));
  TRY(launch_zero(Y, (size_t)(no3 * nv), s));
  TRY(launch_back_transform(L2d, lt, no, nv, s));
  PtrTable pt;
  jac_fill_ptrs(c, &pt);
  pt.p[B_LT] = lt;
  pt.p[B_WS_WR] = wsW;
  pt.p[B_WS_TTR] = wsT;
  pt.p[B_DY] = Y;
  pt.p[B_DVV] = Dvv;
  pt.p[B_DOV] = Dov;
  for (int t0 = 0; t0 < c->ntri; t0 += c->batch) {
    const int t1 = std::min(c->ntri, t0 + c->batch);
    TRY(jac_tau_batch(c, t0, t1, s));  // tau -> ws_w ([c][a][b]), tau~ -> ws_tt
    TRY(left_l3_batch(c, pt, t0, t1, w, L1d, lt, tri, wsW, wsT, s));
    Plan py, pv, pq;
    for (int t = t0; t < t1; ++t) {
      plan_density_occ(py, pv, no, nv, &c->tri_host[3 * t], t - t0);
      plan_left_q(pq, no, nv, &c->tri_host[3 * t], t - t0);
    }
    TRY(jac_run_plan(c, py, 1, pt, s));
    TRY(jac_run_plan(c, pv, 0, pt, s));
    TRY(jac_run_plan(c, pq, 1, pt, s));
  }
  TRY(density_tail(c, pt, Dvv, s));
  TRY(density_virtual(c, pt, w, L1d, lt, Doo, s));
  CU(cudaStreamSynchronize(s));
  return CC3_OK;
}

// C[k][l] += wgt_ij sum_e X_k(e) Y_l(e) over the pairs i >= j (blockIdx.y), with
// X_k the view (i,j,k) of L~ and Y_l the view (i,j,l) of tau, e = (a,b,c) the
// virtual triple of the view.  tab[((y*2 + h)*no + k)*4 + {0..3}] = {T, s0, s1,
// s2}: the stored tensor T ([a][b][c] double-float, T < 0: a zero row) and the
// strides of the view's three slots in it.  Per chunk of DOO_E values of e the
// block stages the 2 no rows (double-float) in shared memory (a padded row
// stride), then each thread accumulates up to 4 of the no^2 products
// (blockIdx.z selects the group of 1024 products) in FP32 arithmetic: each
// double-float product as a rounded high part plus its error and cross terms
// (FMA), the high parts summed with their rounding errors (two-sum), the low
// parts plainly; each chunk's sum then adds into an FP64 accumulator.  The
// terms keep ~2^-44 of their size, well inside the FP64 path's agreement.
constexpr int DOO_E = 128, DOO_LD = DOO_E + 1;
__global__ void __launch_bounds__(256)
    doo_pairs_kernel(const float2 *__restrict__ lt_all, const float2 *__restrict__ tau_all,
                     const long long *__restrict__ tab, const double *__restrict__ wgt, int no,
                     int nv, double *__restrict__ C) {
  extern __shared__ float2 sm2[];  // [2][no][DOO_LD]
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long *tb = tab + (long long)blockIdx.y * 2 * no * 4;
  const int t = threadIdx.x, e0 = t % DOO_E, h = t / DOO_E;  // h: 0 = L~, 1 = tau
  const float2 *X = h ? tau_all : lt_all;
  const int nprod = no * no, pbase = blockIdx.z * 1024;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long nchunk = (nv3 + DOO_E - 1) / DOO_E;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long e = ch * DOO_E + e0;
    const bool in = e < nv3;
    const long long v0 = in ? e / nv2 : 0, v1 = in ? (e / nv) % nv : 0, v2 = in ? e % nv : 0;
    __syncthreads();  // the previous chunk's products are done
    for (int k = 0; k < no; ++k) {
      const long long *r = tb + ((long long)h * no + k) * 4;
      float2 x = make_float2(0.f, 0.f);
      if (in && r[0] >= 0) x = X[r[0] * nv3 + v0 * r[1] + v1 * r[2] + v2 * r[3]];
      sm2[(h * no + k) * DOO_LD + e0] = x;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = pbase + t + 256 * q;
      if (p < nprod) {
        const float2 *xa = sm2 + (p / no) * DOO_LD, *yb = sm2 + (no + p % no) * DOO_LD;
        float shi = 0.f, slo = 0.f;
#pragma unroll 4
        for (int u = 0; u < DOO_E; ++u) {
          const float2 x = xa[u], y = yb[u];
          const float ph = __fmul_rn(x.x, y.x);
          float pl = __fmaf_rn(x.x, y.x, -ph);
          pl = __fmaf_rn(x.x, y.y, pl);
          pl = __fmaf_rn(x.y, y.x, pl);
          const float sn = __fadd_rn(shi, ph);
          const float bb = __fsub_rn(sn, shi);
          const float er = __fadd_rn(__fsub_rn(shi, __fsub_rn(sn, bb)), __fsub_rn(ph, bb));
          shi = sn;
          slo = __fadd_rn(slo, __fadd_rn(er, pl));
        }
        acc[q] += (double)shi + (double)slo;
      }
    }
  }
  const double w = wgt[blockIdx.y];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int p = pbase + t + 256 * q;
    if (p < nprod) atomicAdd(C + p, w * acc[q]);
  }
}

}  // namespace

// Dov[l][d] -= sum_{k,i,c} Y[l][k][i][c] t[k][i][c][d] (pt: B_DY = Y, B_DOV = Dov),
// then Dvv *= 1/2: the end of the occupied loop, on both paths
int density_tail(cc3_ctx *c, const PtrTable &pt, double *Dvv, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv;
  Plan pf;
  // K = no^2 nv over few tiles: split K across CTAs
  const int ks = std::max(1, std::min(128, no * no * nv / 512));
  const int jb = new_job(pf, 0, no, nv, nv, 1, ks, EPI_ATOMIC);
  add_term(pf, jb, op(B_DY, 0, (long long)no * no * nv, 1, 0, 1), op(B_T2, 0, 1, nv),
           no * no * nv);
  const OutD o = out(B_DOV, 0, nv, 1);
  pf.jobs[jb].C = o;
  pf.jobs[jb].Ct = o;
  TRY(jac_run_plan(c, pf, 0, pt, s));
  scale_kernel<<<grid_for(nv2), 256, 0, s>>>(Dvv, nv2, 0.5);
  CU(cudaGetLastError());
  c->counters.launches++;
  return CC3_OK;
}

// Doo[l][k] = -1/2 sum_{ij} sum_{abc} L~^{abc}_{ijk} tau^{abc}_{ijl} from tau and L~ of
// every triple held resident (tau_all, lt_all: [T][a][b][c] double-float, T the
// index in tri of the sorted triple; L~ is zero where i = j = k).  Both tensors are
// symmetric under a simultaneous permutation of occupied and virtual indices, so
// the pair (j, i) gives the same sum over (a,b,c) as (i, j): the pairs i > j count
// twice, i = j once, and one launch covers them all.
int density_doo_resident(cc3_ctx *c, const float2 *tau_all, const float2 *lt_all,
                         const std::vector<int> &tri, double *Doo, cudaStream_t s) {
  const int no = c->no, nv = c->nv;
  const long long nv2 = (long long)nv * nv;
  const int nt = (int)tri.size() / 3;
  std::vector<int> where((size_t)no * no * no, -1);  // sorted triple -> index in tri
  for (int t = 0; t < nt; ++t)
    where[((size_t)tri[3 * t] * no + tri[3 * t + 1]) * no + tri[3 * t + 2]] = t;
  // row of the view (p,q,r): {T, strides of the view's slots in T's storage}
  auto row = [&](int p, int q, int r, bool zero, long long *o) {
    o[0] = -1;
    o[1] = o[2] = o[3] = 0;
    if (zero) return;
    int x[3] = {p, q, r};
    std::sort(x, x + 3, [](int u, int v) { return u > v; });
    const int T = where[((size_t)x[0] * no + x[1]) * no + x[2]];
    if (T < 0) return;
    const long long str[3] = {nv2, nv, 1};
    for (int u = 0; u < 6; ++u) {
      const int *m = PERM6[u];
      const int *tt = &tri[3 * T];
      if (tt[m[0]] == p && tt[m[1]] == q && tt[m[2]] == r) {
        o[0] = T;
        o[1] = str[m[0]];
        o[2] = str[m[1]];
        o[3] = str[m[2]];
        return;
      }
    }
  };
  const int npair = no * (no + 1) / 2;
  std::vector<long long> tab((size_t)npair * 2 * no * 4);
  std::vector<double> wgt(npair);
  int y = 0;
  for (int i = 0; i < no; ++i)
    for (int j = 0; j <= i; ++j, ++y) {
      wgt[y] = i == j ? 1.0 : 2.0;
      for (int k = 0; k < no; ++k) {
        row(i, j, k, i == j && j == k, &tab[(((size_t)y * 2 + 0) * no + k) * 4]);
        row(i, j, k, false, &tab[(((size_t)y * 2 + 1) * no + k) * 4]);
      }
    }
  Bufs B;
  double *C = nullptr, *dw = nullptr;
  long long *dtab = nullptr;
  TRY(B.get(&C, (size_t)no * no));
  TRY(B.get(&dw, (size_t)npair));
  TRY(B.get(&dtab, tab.size()));
  TRY(launch_zero(C, (size_t)no * no, s));
  CU(cudaMemcpyAsync(dtab, tab.data(), sizeof(long long) * tab.size(), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(dw, wgt.data(), sizeof(double) * npair, cudaMemcpyHostToDevice, s));
  const size_t smem = sizeof(float2) * 2 * no * DOO_LD;
  if (smem > 227 * 1024) return CC3_FAIL(CC3_ERR_UNSUPPORTED, "too many occupied orbitals");
  CU(cudaFuncSetAttribute(doo_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem));
  const long long nchunk = (nv2 * nv + DOO_E - 1) / DOO_E;
  int dev = 0, nsm = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int gz = (no * no + 1023) / 1024;
  const long long gx = std::max<long long>(
      1, std::min<long long>(nchunk, (4LL * nsm + (long long)npair * gz - 1) / ((long long)npair * gz)));
  trace_begin(c, TR_FP64_ELEM, s);
  doo_pairs_kernel<<<dim3((unsigned)gx, npair, gz), 256, smem, s>>>(lt_all, tau_all, dtab, dw, no,
                                                                     nv, C);
  CU(cudaGetLastError());
  trace_end(c, TR_FP64_ELEM, s, 2.0 * no * no * (double)npair * nv2 * nv, 0.0);
  c->counters.launches++;
  // Doo[l][k] = -1/2 C[k][l]
  std::vector<double> hc((size_t)no * no), hd((size_t)no * no);
  CU(cudaMemcpyAsync(hc.data(), C, sizeof(double) * no * no, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (int k = 0; k < no; ++k)
    for (int l = 0; l < no; ++l) hd[(size_t)l * no + k] = -0.5 * hc[(size_t)k * no + l];
  CU(cudaMemcpyAsync(Doo, hd.data(), sizeof(double) * no * no, cudaMemcpyHostToDevice, s));
  CU(cudaStreamSynchronize(s));
  return CC3_OK;
}
}  // namespace cc3

extern "C" int cc3_density_triples(cc3_ctx *c, cc3_prec prec, double omega, const double *L1,
                                   const double *L2, double *D_oo, double *D_ov, double *D_vv,
                                   void *cuda_stream) {
  using namespace cc3;
  if (!c || !L1 || !L2 || !D_oo || !D_ov || !D_vv) return CC3_ERR_ARG;
  if (c->general)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "the densities need symmetric integrals");
  if (prec == CC3_SPLIT_INT8) return CC3_FAIL(CC3_ERR_UNSUPPORTED, "no INT8 slice path");
  if (prec != CC3_FP64 && prec != CC3_SPLIT_BF16) return CC3_ERR_ARG;
  if (c->flags & CC3_DETERMINISTIC)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "deterministic reductions cover the residual only");
  if (prec == CC3_FP64 && c->no > DV_MAX_NO)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "the FP64 densities take at most 24 occupied orbitals");
  if (!std::isfinite(omega)) return CC3_FAIL(CC3_ERR_ARG, "non-finite frequency");
  const int no = c->no, nv = c->nv;
  std::lock_guard<std::mutex> lk(c->mu);
  // the occupied loop runs over every triple: a restricted list is refused
  const long long full = (long long)no * (no + 1) * (no + 2) / 6 - no;
  if (c->ntri != full)
    return CC3_FAIL(CC3_ERR_UNSUPPORTED, "the densities need the full triples list");
  {
    // the virtual loop also divides at i = j = k
    std::vector<int> all;
    for (int i = 0; i < no; ++i)
      for (int j = 0; j <= i; ++j)
        for (int k = 0; k <= j; ++k) {
          all.push_back(i);
          all.push_back(j);
          all.push_back(k);
        }
    if (!all.empty() &&
        denominator_gap(no, nv, c->eo_h.data(), c->ev_h.data(), (int)all.size() / 3, all.data(),
                        omega) < CC3_DENOM_MIN)
      return CC3_FAIL(CC3_ERR_DENOM,
                      "the frequency lies within CC3_DENOM_MIN of a triples denominator");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t n1 = (size_t)no * nv, nt2 = n1 * no * nv, noo = (size_t)no * no,
               nvv = (size_t)nv * nv;
  c->counters = cc3_counters{};
  trace_reset(c);
  {
    const double v4 = (double)nv * nv * nv * nv, o3 = (double)no * no * no;
    const double nvt = (double)nv * (nv + 1) * (nv + 2) / 6.0 - nv;
    c->counters.nominal_flop = 6.0 * v4 * (o3 - no) + 24.0 * nv * o3 * nvt;
  }
  const bool dev = (c->flags & CC3_DEVICE_PTRS) != 0;
  double *dL1 = const_cast<double *>(L1), *dL2 = const_cast<double *>(L2), *doo = D_oo,
         *dov = D_ov, *dvv = D_vv;
  std::vector<double *> tmp;
  auto mk = [&](double **p, size_t n) {
    if (cudaMalloc(p, sizeof(double) * (n ? n : 1)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    tmp.push_back(*p);
    return true;
  };
  int rc = CC3_OK;
  if (!dev) {
    if (!mk(&dL1, n1) || !mk(&dL2, nt2) || !mk(&doo, noo) || !mk(&dov, n1) || !mk(&dvv, nvv))
      rc = CC3_FAIL(CC3_ERR_OOM, "density staging");
    if (rc == CC3_OK &&
        (cudaMemcpyAsync(dL1, L1, sizeof(double) * n1, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(dL2, L2, sizeof(double) * nt2, cudaMemcpyHostToDevice, s) != cudaSuccess))
      rc = CC3_FAIL(CC3_ERR_CUDA, "density upload");
  }
  if (rc == CC3_OK)
    rc = prec == CC3_SPLIT_BF16 ? split_density(c, omega, dL1, dL2, doo, dov, dvv, s)
                                : density_fp64(c, omega, dL1, dL2, doo, dov, dvv, s);
  if (rc == CC3_OK && !dev) {
    if (cudaMemcpyAsync(D_oo, doo, sizeof(double) * noo, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(D_ov, dov, sizeof(double) * n1, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(D_vv, dvv, sizeof(double) * nvv, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = CC3_FAIL(CC3_ERR_CUDA, "density download");
  }
  cudaStreamSynchronize(s);
  for (double *p : tmp) cudaFree(p);
  if (rc == CC3_OK) rc = trace_collect(c, s);
  return rc;
}
