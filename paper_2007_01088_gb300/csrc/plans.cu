// Host-side construction of contraction job lists for the FP64 engine.
//
// Triples amplitudes (paper, Algorithm 1, the tau amplitudes, and eq. "permutation"):
//   W^{abc}_{ijk} = P^{abc}_{ijk} B,  B^{xyz}_{pqr} = sum_d t^{xd}_{pq} gv_{ydzr}
//                                                  - sum_l t^{xy}_{pl} go_{lqzr}
// with gv[y][d][z][r] the vvvo block and go[l][q][z][r] the oovo block (both
// in general, non-symmetric form so that the Jacobian's R1-dressed blocks use
// the same jobs).  The six P terms (ordered triples with their virtual slots)
// are split over two tile shapes that write the same layout W[c][a][b]:
//   phase AB, tile (a, b) at fixed c: the four terms whose t-row index is a
//     or b, plus the four occupied terms whose integral index z is a or b;
//   phase C, tile (c, (a,b)): the two terms whose t-row index is c and the
//     two occupied terms with z = c; its epilogue divides by (w - eps).
// Residual contractions (Algorithm 1, "for permutations of i,j,k"): for each
// distinct ordered (p,q,r) = (ijk[s0], ijk[s1], ijk[s2]) the amplitude
// tau~^{xyz}_{pqr} is tau~_{ijk} with x in slot s0, y in s1, z in s2, read
// through strides (no reordered copy).
#include <algorithm>

#include "cc3_internal.h"

namespace cc3 {

static const int BIG = 1 << 30;

Opnd op(int buf, long long off, long long sm0, long long sk0, long long sb, int neg) {
  Opnd o;
  o.buf = buf;
  o.m_in = BIG;
  o.k_in = BIG;
  o.neg = neg;
  o.off = off;
  o.sb = sb;
  o.sm1 = 0;
  o.sm0 = sm0;
  o.sk1 = 0;
  o.sk0 = sk0;
  return o;
}
Opnd with_m2(Opnd o, int m_in, long long sm1) {
  o.m_in = m_in;
  o.sm1 = sm1;
  return o;
}
Opnd with_k2(Opnd o, int k_in, long long sk1) {
  o.k_in = k_in;
  o.sk1 = sk1;
  return o;
}
OutD out(int buf, long long off, long long sm0, long long sn0, long long sb) {
  OutD c;
  c.buf = buf;
  c.m_in = BIG;
  c.n_in = BIG;
  c.off = off;
  c.sb = sb;
  c.sm1 = 0;
  c.sm0 = sm0;
  c.sn1 = 0;
  c.sn0 = sn0;
  return c;
}

static void tile_dims(int kind, int *BM, int *BN) {
  if (kind == 0) { *BM = 64; *BN = 64; }
  else { *BM = 256; *BN = 4; }
}

// Appends a job; returns its index.  Terms are appended with add_term.
int new_job(Plan &P, int kind, int M, int N, int Nm, int batch, int ksplit, int mode) {
  int BM, BN;
  tile_dims(kind, &BM, &BN);
  Job j{};
  j.M = M;
  j.N = N;
  j.Nm = Nm;
  j.batch = batch;
  j.ksplit = std::max(1, ksplit);
  j.mode = mode;
  j.tiles_m = (M + BM - 1) / BM;
  j.tiles_n = (N + BN - 1) / BN;
  j.tile_base = P.tiles;
  j.term0 = (int)P.terms.size();
  j.nterm = 0;
  j.C = out(B_SCRATCH, 0, 0, 0);
  j.Ct = j.C;
  P.tiles += (long long)batch * j.tiles_m * j.tiles_n * j.ksplit;
  P.jobs.push_back(j);
  return (int)P.jobs.size() - 1;
}
void add_term(Plan &P, int job, const Opnd &A, const Opnd &B, int K, const Opnd *Bt) {
  Term t;
  t.A = A;
  t.B = B;
  t.Bt = Bt ? *Bt : B;
  t.K = K;
  P.terms.push_back(t);
  P.jobs[job].nterm++;
}

// --- W build -----------------------------------------------------------------
// Adds the terms of one (t, gv, go) set to the AB job (phase 0) or the C job
// (phase 1) of triple (i,j,k).
static void w_terms(Plan &P, int job, int phase, int no, int nv, int i, int j,
                    int k, int bt, int bv, int bo) {
  const long long nv2 = (long long)nv * nv, nvo = (long long)nv * no;
  const long long v2o = nv2 * no, o2v = (long long)no * no * nv;
  auto tpq = [&](int p, int q) { return ((long long)p * no + q) * nv2; };
  auto trow = [&](int p, int q) { return op(bt, tpq(p, q), nv, 1); };  // t[p][q][x][d], rows x
  if (phase == 0) {  // tile (a, b) at fixed c = batch index
    // (i,j,k): sum_d t_ij[a][d] gv[b][d][c][k]
    add_term(P, job, trow(i, j), op(bv, k, v2o, nvo, no), nv);
    // (i,k,j): sum_d t_ik[a][d] gv[c][d][b][j]
    add_term(P, job, trow(i, k), op(bv, j, no, nvo, v2o), nv);
    // (j,i,k): sum_d gv[a][d][c][k] t_ji[b][d]
    add_term(P, job, op(bv, k, v2o, nvo, no), trow(j, i), nv);
    // (j,k,i): sum_d gv[c][d][a][i] t_jk[b][d]
    add_term(P, job, op(bv, i, no, nvo, v2o), trow(j, k), nv);
    // occupied terms, go[l][q][z][r] at ((l*no+q)*nv+z)*no+r
    // (j,k,i): - sum_l go[l][k][a][i] t[j][l][b][c]
    add_term(P, job, op(bo, (long long)k * nvo + i, no, o2v, 0, 1),
             op(bt, (long long)j * no * nv2, nv, nv2, 1), no);
    // (k,j,i): - sum_l go[l][j][a][i] t[k][l][c][b]
    add_term(P, job, op(bo, (long long)j * nvo + i, no, o2v, 0, 1),
             op(bt, (long long)k * no * nv2, 1, nv2, nv), no);
    // (k,i,j): - sum_l t[k][l][c][a] go[l][i][b][j]
    add_term(P, job, op(bt, (long long)k * no * nv2, 1, nv2, nv, 1),
             op(bo, (long long)i * nvo + j, no, o2v), no);
    // (i,k,j): - sum_l t[i][l][a][c] go[l][k][b][j]
    add_term(P, job, op(bt, (long long)i * no * nv2, nv, nv2, 1, 1),
             op(bo, (long long)k * nvo + j, no, o2v), no);
  } else {  // tile (c, (a,b)), n = a*nv + b
    // (k,i,j): sum_d t_ki[c][d] gv[a][d][b][j]
    add_term(P, job, trow(k, i), with_m2(op(bv, j, no, nvo), nv, v2o), nv);
    // (k,j,i): sum_d t_kj[c][d] gv[b][d][a][i]
    add_term(P, job, trow(k, j), with_m2(op(bv, i, v2o, nvo), nv, no), nv);
    // (i,j,k) occupied: - sum_l go[l][j][c][k] t[i][l][a][b]
    add_term(P, job, op(bo, (long long)j * nvo + k, no, o2v, 0, 1),
             with_m2(op(bt, (long long)i * no * nv2, 1, nv2), nv, nv), no);
    // (j,i,k) occupied: - sum_l go[l][i][c][k] t[j][l][b][a]
    add_term(P, job, op(bo, (long long)i * nvo + k, no, o2v, 0, 1),
             with_m2(op(bt, (long long)j * no * nv2, nv, nv2), nv, 1), no);
  }
}

void plan_w_build(Plan &P, int no, int nv, const int ijk[3], int slot,
                  int buf_w, const TermSet *sets, int nsets, double w,
                  double eo, int phase) {
  // phase 0: AB job (store into W[slot][c][a][b]); phase 1: C job, whose
  // epilogue forms tau = W / (w - eps) in place.  Several (t, gv, go) sets
  // add up (the Jacobian's R3 = P(R2, g) + P(t2, g^)).
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  if (phase == 0) {
    int jb = new_job(P, 0, nv, nv, nv, nv, 1, EPI_STORE);
    P.jobs[jb].C = out(buf_w, slot * nv3, nv, 1, nv2);
    for (int s = 0; s < nsets; ++s)
      w_terms(P, jb, 0, no, nv, i, j, k, sets[s].bt, sets[s].bv, sets[s].bo);
  } else {
    int jb = new_job(P, 0, nv, (int)nv2, (int)nv2, 1, 1, EPI_TAU);
    OutD c = out(buf_w, slot * nv3, nv2, 1);
    c.n_in = nv;
    c.sn1 = nv;
    P.jobs[jb].C = c;
    P.jobs[jb].w = w;
    P.jobs[jb].eo = eo;
    for (int s = 0; s < nsets; ++s)
      w_terms(P, jb, 1, no, nv, i, j, k, sets[s].bt, sets[s].bv, sets[s].bo);
  }
}

// --- residual contractions ----------------------------------------------------
// which: bit 0 = vvov + singles job (64x64 tiles), bit 1 = ooov + F job (thin),
//        bit 2 = F-only job (thin; Jacobian tau~ . F^ term), bit 3 = leave out
//        the singles and F tail columns of the first two (the left
//        transformation's sigma2 contractions).
void plan_omega_contractions(Plan &P, int no, int nv, const int ijk[3],
                             int slot, int buf_tt, int buf_ovov, int buf_fov,
                             int buf_ooov, bool vvov_from_vvvo, int buf_vvov,
                             int buf_omt, int buf_om1, int ksplit, int which) {
  static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                  {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long st[3] = {nv2, nv, 1};  // tau~[a][b][c] slot strides
  int seen[6][3];
  int nseen = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return;
  for (int s = 0; s < 6; ++s) {
    const int *m = PERM6[s];
    const int p = ijk[m[0]], q = ijk[m[1]], r = ijk[m[2]];
    bool dup = false;
    for (int u = 0; u < nseen; ++u)
      if (seen[u][0] == p && seen[u][1] == q && seen[u][2] == r) dup = true;
    if (dup) continue;
    seen[nseen][0] = p;
    seen[nseen][1] = q;
    seen[nseen][2] = r;
    ++nseen;
    const long long tt0 = slot * nv3;
    if (which & 1) {
      // Omega~^{ad}_{pq} += sum_{yz} V[x][y][z] vvov[d][y][r][z]   (N = nv)
      // Omega1^x_p       += sum_{yz} V[x][y][z] ovov[q][y][r][z]   (tail col)
      int jb = new_job(P, 0, nv, (which & 8) ? nv : nv + 1, nv, 1, ksplit, EPI_ATOMIC);
      Opnd A = with_k2(op(buf_tt, tt0, st[m[0]], st[m[2]]), nv, st[m[1]]);
      Opnd B;
      if (vvov_from_vvvo)  // vvov[d][y][r][z] = vvvo[y][d][z][r]
        B = with_k2(op(buf_vvov, r, (long long)nv * no, no), nv, nv2 * no);
      else  // vvov[d][b][k][c]
        B = with_k2(op(buf_vvov, (long long)r * nv, nv2 * no, 1), nv,
                    (long long)no * nv);
      Opnd Bt = with_k2(op(buf_ovov, (long long)q * nv * no * nv + (long long)r * nv, 0, 1),
                        nv, (long long)no * nv);
      add_term(P, jb, A, B, (int)nv2, &Bt);
      P.jobs[jb].C = out(buf_omt, ((long long)p * no + q) * nv2, nv, 1);
      P.jobs[jb].Ct = out(buf_om1, (long long)p * nv, 1, 0);
    }
    if (which & 2) {
      // Omega~^{xy}_{pl} -= sum_z V[x][y][z] ooov[q][l][r][z]     (N = no)
      // Omega~^{xy}_{pq} += sum_z V[x][y][z] F[r][z]              (tail col)
      int jb = new_job(P, 1, (int)nv2, (which & 8) ? no : no + 1, no, 1, 1, EPI_ATOMIC);
      Opnd A = with_m2(op(buf_tt, tt0, st[m[1]], st[m[2]]), nv, st[m[0]]);
      Opnd B = op(buf_ooov, (long long)q * no * no * nv + (long long)r * nv,
                  (long long)no * nv, 1, 0, 1);
      Opnd Bt = op(buf_fov, (long long)r * nv, 0, 1);
      add_term(P, jb, A, B, nv, &Bt);
      OutD c = out(buf_omt, (long long)p * no * nv2, 1, nv2);
      c.m_in = nv;
      c.sm1 = nv;
      P.jobs[jb].C = c;
      OutD ct = out(buf_omt, ((long long)p * no + q) * nv2, 1, 0);
      ct.m_in = nv;
      ct.sm1 = nv;
      P.jobs[jb].Ct = ct;
    }
    if (which & 4) {
      // Omega~^{xy}_{pq} += sum_z V[x][y][z] F[r][z]  only
      int jb = new_job(P, 1, (int)nv2, 1, 0, 1, 1, EPI_ATOMIC);
      Opnd A = with_m2(op(buf_tt, tt0, st[m[1]], st[m[2]]), nv, st[m[0]]);
      Opnd Bt = op(buf_fov, (long long)r * nv, 0, 1);
      add_term(P, jb, A, Bt, nv, &Bt);
      OutD ct = out(buf_omt, ((long long)p * no + q) * nv2, 1, 0);
      ct.m_in = nv;
      ct.sm1 = nv;
      P.jobs[jb].C = ct;
      P.jobs[jb].Ct = ct;
    }
  }
}

double nominal_flop_omega(int no, int nv, int nperm_total) {
  // 4 nv^4 per distinct ordered triple (2 for the W build, 2 for the vvov
  // contraction); over all triples this is 4 nv^4 (no^3 - no)
  (void)no;
  return 4.0 * (double)nv * nv * nv * nv * (double)nperm_total;
}

}  // namespace cc3
