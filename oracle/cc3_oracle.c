/*
 * Plain FP64 CPU oracle for the closed-shell CC3 triples hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the GPU path.
 *
 * What it computes (Paul, Myhre, Koch, "A new and efficient implementation of
 * CC3", arXiv 2007.01088, section "Implementation"):
 *
 *   oracle_omega      Algorithm 1 (CC3 ground-state triples residual): the
 *                     restricted loop i >= j >= k, the permutation operator
 *                     P^{abc}_{ijk} (eq. "permutation"), the orbital-energy
 *                     denominator, the contravariant combination of Algorithm 1,
 *                     the four contractions for every distinct permutation of
 *                     (i,j,k), and the back-transform (1/3) P^{ab}_{ij}(2X+X^{ba}).
 *   oracle_prep       Algorithm 2 (Z^v and Z^o intermediates).
 *   oracle_left_jacobian  The left (transpose) Jacobian transformation: the
 *                     covariant L3 amplitudes, their contravariant form and
 *                     their contractions, read as the exact transpose of the
 *                     right transformation below.
 *   oracle_jacobian   The right CC3 Jacobian transformation of trial vectors,
 *                     reconstructed from eq. "jcc3": R3 = (w - eps)^{-1}
 *                     <mu3|[H,R2] + [[H,R1],T2]>, rho = <mu1|[H,R3]> and
 *                     <mu2|[H,R3]> + <mu2|[[H,R1],T3]>, with the R1-dressed
 *                     integrals from the first-order T1 transformation.
 *
 * The integrals enter in the general five-block form, so that the same code
 * serves T1-transformed (non-symmetric) integrals:
 *   vvvo[b][d][c][k] = g_{bdck}     oovo[l][j][c][k] = g_{ljck}
 *   ooov[j][l][k][c] = g_{jlkc}     ovov[j][b][k][c] = g_{jbkc}
 *   vvov[d][b][k][c] = g_{dbkc}     F_ov[k][c]
 * and t2[i][j][a][b] = t^{ab}_{ij}, omega1[i][a], omega2[i][j][a][b].
 *
 * Readings of the paper taken here (the paper is silent or garbled there):
 *  - The contravariant amplitudes permute the virtual indices with i,j,k fixed
 *    (Algorithm 1 form); eq. "contra_t" as printed permutes both index sets.
 *  - "For permutations of i,j,k" runs over the DISTINCT ordered triples
 *    (6, 3 or 0 of them); for (p,q,r) = (ijk[s0], ijk[s1], ijk[s2]) the
 *    amplitude tau^{xyz}_{pqr} is the element of tau_{ijk} that holds x in slot
 *    s0, y in slot s1 and z in slot s2 (each virtual index travels with its
 *    occupied partner, by the six-fold symmetry).
 *  - P^{ab}_{ij} X^{ab}_{ij} = X^{ab}_{ij} + X^{ba}_{ji} in the back-transform.
 *  - The triples energy is E_T = sum_{ijab} t^{ab}_{ij} Omega~^{ab}_{ij}.
 *  - tau = -W / eps with eps^{abc}_{ijk} = e_a+e_b+e_c-e_i-e_j-e_k (plain
 *    orbital energies); the R3 denominator is (w - eps)^{-1}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Parallel work split.  The triple loops run one triple per thread when
 * there are at least as many triples as threads; with fewer triples the loop
 * runs in one thread and the loops over the first virtual index inside each
 * step are split over the threads instead (each thread then owns whole rows
 * of the arrays it writes, so every element is summed in the same order
 * either way). */
#ifdef _OPENMP
#define ORACLE_PRAGMA(x) _Pragma(#x)
#define ORACLE_INNER_FOR ORACLE_PRAGMA(omp parallel for if (!omp_in_parallel()) schedule(static))
#else
#define ORACLE_INNER_FOR
#endif

typedef struct {
  int no, nv;
  const double *eps_o, *eps_v, *t2;
  const double *vvvo, *oovo, *ooov, *ovov, *vvov, *F_ov;
} blocks_t;

#define T2(B, i, j, a, b) (B)->t2[(((size_t)(i) * (B)->no + (j)) * (B)->nv + (a)) * (B)->nv + (b)]
#define VVVO(B, b, d, c, k) (B)->vvvo[(((size_t)(b) * (B)->nv + (d)) * (B)->nv + (c)) * (B)->no + (k)]
#define OOVO(B, l, j, c, k) (B)->oovo[(((size_t)(l) * (B)->no + (j)) * (B)->nv + (c)) * (B)->no + (k)]
#define OOOV(B, j, l, k, c) (B)->ooov[(((size_t)(j) * (B)->no + (l)) * (B)->no + (k)) * (B)->nv + (c)]
#define OVOV(B, j, b, k, c) (B)->ovov[(((size_t)(j) * (B)->nv + (b)) * (B)->no + (k)) * (B)->nv + (c)]
#define VVOV(B, d, b, k, c) (B)->vvov[(((size_t)(d) * (B)->nv + (b)) * (B)->no + (k)) * (B)->nv + (c)]

/* The six terms of the permutation operator P^{abc}_{ijk}: term s puts the
 * ordered occupied triple (ijk[s0], ijk[s1], ijk[s2]) with virtual indices
 * (v[s0], v[s1], v[s2]), v = (a,b,c).  Order as in eq. "permutation":
 * B^{abc}_{ijk} + B^{bac}_{jik} + B^{cba}_{kji} + B^{acb}_{ikj} + B^{bca}_{jki}
 * + B^{cab}_{kij}. */
static const int PERM6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0},
                                {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};

/* B_{pqr}[x][y][z] = sum_d t^{xd}_{pq} g_{ydzr} - sum_l t^{xy}_{pl} g_{lqzr}
 * (the bracket that defines tau in Algorithms 1 and 2, for one ordered triple).
 * t and the two integral blocks are passed separately so that the Jacobian can
 * call the same builder with (R2, g) and (t2, g-hat). */
static void build_B(int no, int nv, const double *t, const double *gvvvo,
                    const double *goovo, int p, int q, int r, double *Bout,
                    long long *flops) {
  size_t nv2 = (size_t)nv * nv;
  /* each element B[x][y][z] is the sum over d in increasing order, then the
   * l terms in increasing order; the z loop is innermost so that the
   * integral block is read along its rows */
  ORACLE_INNER_FOR
  for (int x = 0; x < nv; ++x)
    for (int y = 0; y < nv; ++y) {
      double *row = Bout + (size_t)x * nv2 + (size_t)y * nv;
      const double *tr = t + (((size_t)p * no + q) * nv + x) * nv;
      for (int z = 0; z < nv; ++z) row[z] = 0.0;
      for (int d = 0; d < nv; ++d) {
        const double td = tr[d];
        const double *g = gvvvo + ((size_t)y * nv + d) * nv * no + r;
        for (int z = 0; z < nv; ++z) row[z] += td * g[(size_t)z * no];
      }
      for (int l = 0; l < no; ++l) {
        const double tl = t[(((size_t)p * no + l) * nv + x) * nv + y];
        const double *g = goovo + ((size_t)l * no + q) * nv * no + r;
        for (int z = 0; z < nv; ++z) row[z] -= tl * g[(size_t)z * no];
      }
    }
  /* dominant term only: the d-sum is one nv x nv^2 x nv contraction */
  if (flops) *flops += 2LL * nv * nv * nv * nv;
}

/* W = P^{abc}_{ijk} B for one unique triple; each distinct ordered triple's B
 * is built once and placed in every slot arrangement P asks for. */
static void build_W(int no, int nv, const double *t, const double *gvvvo,
                    const double *goovo, const int ijk[3], double *W,
                    double *Bscratch, long long *flops) {
  size_t nv2 = (size_t)nv * nv, nv3 = nv2 * nv;
  memset(W, 0, nv3 * sizeof(double));
  int done[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < 6; ++s) {
    if (done[s]) continue;
    int p = ijk[PERM6[s][0]], q = ijk[PERM6[s][1]], r = ijk[PERM6[s][2]];
    build_B(no, nv, t, gvvvo, goovo, p, q, r, Bscratch, flops);
    for (int s2 = s; s2 < 6; ++s2) {
      if (ijk[PERM6[s2][0]] != p || ijk[PERM6[s2][1]] != q ||
          ijk[PERM6[s2][2]] != r)
        continue;
      done[s2] = 1;
      const int *m = PERM6[s2];
      ORACLE_INNER_FOR
      for (int v0 = 0; v0 < nv; ++v0) {
        int v[3];
        v[0] = v0;
        for (v[1] = 0; v[1] < nv; ++v[1])
          for (v[2] = 0; v[2] < nv; ++v[2]) {
            size_t src = (size_t)v[m[0]] * nv2 + (size_t)v[m[1]] * nv + v[m[2]];
            W[(size_t)v[0] * nv2 + (size_t)v[1] * nv + v[2]] += Bscratch[src];
          }
      }
    }
  }
}

/* tau~^{abc} = 4 tau^{abc} - 2 tau^{acb} - 2 tau^{cba} - 2 tau^{bac}
 *              + tau^{bca} + tau^{cab}      (Algorithm 1, i,j,k fixed) */
static void contravariant(int nv, const double *tau, double *tt) {
  size_t nv2 = (size_t)nv * nv;
#define TAU(a, b, c) tau[(size_t)(a) * nv2 + (size_t)(b) * nv + (c)]
  ORACLE_INNER_FOR
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b)
      for (int c = 0; c < nv; ++c)
        tt[(size_t)a * nv2 + (size_t)b * nv + c] =
            4.0 * TAU(a, b, c) - 2.0 * TAU(a, c, b) - 2.0 * TAU(c, b, a) -
            2.0 * TAU(b, a, c) + TAU(b, c, a) + TAU(c, a, b);
#undef TAU
}

/* The distinct ordered permutations of (i,j,k): returns how many (6, 3 or 0)
 * and, for each, the slot map s (p,q,r) = (ijk[s0], ijk[s1], ijk[s2]). */
static int distinct_perms(const int ijk[3], int maps[6][3]) {
  int n = 0;
  if (ijk[0] == ijk[1] && ijk[1] == ijk[2]) return 0;
  for (int s = 0; s < 6; ++s) {
    int p = ijk[PERM6[s][0]], q = ijk[PERM6[s][1]], r = ijk[PERM6[s][2]];
    int seen = 0;
    for (int u = 0; u < n; ++u)
      if (ijk[maps[u][0]] == p && ijk[maps[u][1]] == q && ijk[maps[u][2]] == r)
        seen = 1;
    if (!seen) {
      maps[n][0] = PERM6[s][0];
      maps[n][1] = PERM6[s][1];
      maps[n][2] = PERM6[s][2];
      ++n;
    }
  }
  return n;
}

/* View V[x][y][z] = tau~^{xyz}_{pqr} taken from tau~_{ijk}: x sits in slot
 * m[0], y in slot m[1], z in slot m[2]. */
static void permuted_view(int nv, const double *tt, const int m[3], double *V) {
  size_t nv2 = (size_t)nv * nv;
  ORACLE_INNER_FOR
  for (int x = 0; x < nv; ++x)
    for (int y = 0; y < nv; ++y)
      for (int z = 0; z < nv; ++z) {
        int s[3];
        s[m[0]] = x;
        s[m[1]] = y;
        s[m[2]] = z;
        V[(size_t)x * nv2 + (size_t)y * nv + z] =
            tt[(size_t)s[0] * nv2 + (size_t)s[1] * nv + s[2]];
      }
}

/* The four contractions of Algorithm 1 for one ordered triple (p,q,r):
 *   Om1^a_p      += sum_{bc} V^{abc} g_{qbrc}
 *   Om~^{ab}_{pq} += sum_c  V^{abc} F_{rc}
 *   Om~^{ab}_{pl} -= sum_c  V^{abc} g_{qlrc}
 *   Om~^{ad}_{pq} += sum_bc V^{abc} g_{dbrc}                                  */
static void contract_omega(const blocks_t *B, const double *V, int p, int q,
                           int r, double *om1, double *omt, long long *flops) {
  int no = B->no, nv = B->nv;
  size_t nv2 = (size_t)nv * nv;
  ORACLE_INNER_FOR
  for (int a = 0; a < nv; ++a) {
    double s1 = 0.0;
    for (int b = 0; b < nv; ++b)
      for (int c = 0; c < nv; ++c)
        s1 += V[(size_t)a * nv2 + (size_t)b * nv + c] * OVOV(B, q, b, r, c);
    om1[(size_t)p * nv + a] += s1;
  }
  ORACLE_INNER_FOR
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      const double *vr = V + (size_t)a * nv2 + (size_t)b * nv;
      double sF = 0.0;
      for (int c = 0; c < nv; ++c) sF += vr[c] * B->F_ov[(size_t)r * nv + c];
      omt[(((size_t)p * no + q) * nv + a) * nv + b] += sF;
      for (int l = 0; l < no; ++l) {
        double so = 0.0;
        for (int c = 0; c < nv; ++c) so += vr[c] * OOOV(B, q, l, r, c);
        omt[(((size_t)p * no + l) * nv + a) * nv + b] -= so;
      }
    }
  ORACLE_INNER_FOR
  for (int a = 0; a < nv; ++a)
    for (int d = 0; d < nv; ++d) {
      double s = 0.0;
      for (int b = 0; b < nv; ++b)
        for (int c = 0; c < nv; ++c)
          s += V[(size_t)a * nv2 + (size_t)b * nv + c] * VVOV(B, d, b, r, c);
      omt[(((size_t)p * no + q) * nv + a) * nv + d] += s;
    }
  if (flops) *flops += 2LL * nv * nv * nv * nv;
}

/* Denominator (w - eps^{abc}_{ijk}); tau = W / (w - eps), so w = 0 gives the
 * tau of Algorithm 1, tau = -W / eps. */
static void divide_denominator(const blocks_t *B, const int ijk[3], double w,
                               const double *W, double *tau) {
  int nv = B->nv;
  size_t nv2 = (size_t)nv * nv;
  double eo = B->eps_o[ijk[0]] + B->eps_o[ijk[1]] + B->eps_o[ijk[2]];
  ORACLE_INNER_FOR
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b)
      for (int c = 0; c < nv; ++c) {
        double e = B->eps_v[a] + B->eps_v[b] + B->eps_v[c] - eo;
        size_t x = (size_t)a * nv2 + (size_t)b * nv + c;
        tau[x] = W[x] / (w - e);
      }
}

/* Omega2 = (1/3) P^{ab}_{ij} (2 Om~^{ab}_{ij} + Om~^{ba}_{ij}) */
static void back_transform(int no, int nv, const double *omt, double *om2) {
#define OT(i, j, a, b) omt[(((size_t)(i) * no + (j)) * nv + (a)) * nv + (b)]
  for (int i = 0; i < no; ++i)
    for (int j = 0; j < no; ++j)
      for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b)
          om2[(((size_t)i * no + j) * nv + a) * nv + b] =
              (2.0 * OT(i, j, a, b) + OT(i, j, b, a) + 2.0 * OT(j, i, b, a) +
               OT(j, i, a, b)) / 3.0;
#undef OT
}

static int list_triples(int no, int ntri, const int *tri, int **out) {
  if (tri) {
    *out = (int *)malloc(sizeof(int) * 3 * (size_t)(ntri > 0 ? ntri : 1));
    if (!*out) return -1;
    memcpy(*out, tri, sizeof(int) * 3 * (size_t)ntri);
    return ntri;
  }
  int n = 0;
  *out = (int *)malloc(sizeof(int) * 3 * ((size_t)no * no * no + 1));
  if (!*out) return -1;
  for (int i = 0; i < no; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k) {
        if (i == j && j == k) continue;
        (*out)[3 * n] = i;
        (*out)[3 * n + 1] = j;
        (*out)[3 * n + 2] = k;
        ++n;
      }
  return n;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* Algorithm 1.  tri = NULL runs every triple i >= j >= k; otherwise the ntri
 * triples listed (each i >= j >= k) -- the same restriction the GPU library
 * takes.  omega1[no][nv], omega2[no][no][nv][nv], omega2_tilde (may be NULL),
 * E_T (may be NULL).  flops counts the dominant contractions only (the d-sum
 * of each distinct B and the vvov contraction of each distinct permutation).  Returns threads used. */
int oracle_omega(int no, int nv, const double *eps_o, const double *eps_v,
                 const double *t2, const double *vvvo, const double *oovo,
                 const double *ooov, const double *ovov, const double *vvov,
                 const double *F_ov, int ntri, const int *tri, double *omega1,
                 double *omega2, double *omega2_tilde, double *E_T,
                 long long *flops, int nthreads) {
  blocks_t B = {no, nv, eps_o, eps_v, t2, vvvo, oovo, ooov, ovov, vvov, F_ov};
  size_t nv3 = (size_t)nv * nv * nv, n1 = (size_t)no * nv,
         n2 = (size_t)no * no * nv * nv;
  int *T = NULL;
  int nt = list_triples(no, ntri, tri, &T);
  if (nt < 0) return -1;
  int used = set_threads(nthreads);
  double *om1 = (double *)calloc(n1 ? n1 : 1, sizeof(double));
  double *omt = (double *)calloc(n2 ? n2 : 1, sizeof(double));
  long long fl = 0;
#pragma omp parallel if (nt >= used) reduction(+ : fl)
  {
    double *W = (double *)malloc(nv3 * sizeof(double));
    double *S = (double *)malloc(nv3 * sizeof(double));
    double *tau = (double *)malloc(nv3 * sizeof(double));
    double *V = (double *)malloc(nv3 * sizeof(double));
    double *m1 = (double *)calloc(n1 ? n1 : 1, sizeof(double));
    double *mt = (double *)calloc(n2 ? n2 : 1, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < nt; ++t) {
      const int *ijk = T + 3 * t;
      int maps[6][3];
      int np = distinct_perms(ijk, maps);
      if (np == 0) continue;
      build_W(no, nv, t2, vvvo, oovo, ijk, W, S, &fl);
      divide_denominator(&B, ijk, 0.0, W, tau);
      contravariant(nv, tau, S); /* S = tau~ */
      for (int u = 0; u < np; ++u) {
        permuted_view(nv, S, maps[u], V);
        contract_omega(&B, V, ijk[maps[u][0]], ijk[maps[u][1]],
                       ijk[maps[u][2]], m1, mt, &fl);
      }
    }
#pragma omp critical
    {
      for (size_t x = 0; x < n1; ++x) om1[x] += m1[x];
      for (size_t x = 0; x < n2; ++x) omt[x] += mt[x];
    }
    free(W); free(S); free(tau); free(V); free(m1); free(mt);
  }
  if (omega1) memcpy(omega1, om1, n1 * sizeof(double));
  if (omega2) back_transform(no, nv, omt, omega2);
  if (omega2_tilde) memcpy(omega2_tilde, omt, n2 * sizeof(double));
  if (E_T) {
    double e = 0.0;
    for (size_t x = 0; x < n2; ++x) e += t2[x] * omt[x];
    *E_T = e;
  }
  if (flops) *flops = fl;
  free(om1); free(omt); free(T);
  return used;
}

/* Algorithm 2: Z~v[a][b][i][d] -= sum_c tau~^{abc}_{ijk} g_{jdkc} and
 * Z~o[a][j][i][l] += sum_bc tau~^{abc}_{ijk} g_{lbkc}, over every distinct
 * permutation of each triple (ooov here is g_{jdkc} read as ovov[j][d][k][c],
 * the same integrals as the ground state's singles contraction).
 * Zv[nv][nv][no][nv], Zo[nv][no][no][no].  Returns threads used. */
int oracle_prep(int no, int nv, const double *eps_o, const double *eps_v,
                const double *t2, const double *vvvo, const double *oovo,
                const double *ovov, int ntri, const int *tri, double *Zv,
                double *Zo, long long *flops, int nthreads) {
  blocks_t B = {no, nv, eps_o, eps_v, t2, vvvo, oovo, NULL, ovov, NULL, NULL};
  size_t nv3 = (size_t)nv * nv * nv;
  size_t nzv = nv3 * no, nzo = (size_t)nv * no * no * no;
  int *T = NULL;
  int nt = list_triples(no, ntri, tri, &T);
  if (nt < 0) return -1;
  int used = set_threads(nthreads);
  memset(Zv, 0, nzv * sizeof(double));
  memset(Zo, 0, nzo * sizeof(double));
  long long fl = 0;
#pragma omp parallel if (nt >= used) reduction(+ : fl)
  {
    double *W = (double *)malloc(nv3 * sizeof(double));
    double *S = (double *)malloc(nv3 * sizeof(double));
    double *tau = (double *)malloc(nv3 * sizeof(double));
    double *V = (double *)malloc(nv3 * sizeof(double));
    double *zv = (double *)calloc(nzv ? nzv : 1, sizeof(double));
    double *zo = (double *)calloc(nzo ? nzo : 1, sizeof(double));
    size_t nv2 = (size_t)nv * nv;
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < nt; ++t) {
      const int *ijk = T + 3 * t;
      int maps[6][3];
      int np = distinct_perms(ijk, maps);
      if (np == 0) continue;
      build_W(no, nv, t2, vvvo, oovo, ijk, W, S, &fl);
      divide_denominator(&B, ijk, 0.0, W, tau);
      contravariant(nv, tau, S);
      for (int u = 0; u < np; ++u) {
        int p = ijk[maps[u][0]], q = ijk[maps[u][1]], r = ijk[maps[u][2]];
        permuted_view(nv, S, maps[u], V);
        ORACLE_INNER_FOR
        for (int a = 0; a < nv; ++a)
          for (int b = 0; b < nv; ++b)
            for (int d = 0; d < nv; ++d) {
              double s = 0.0;
              for (int c = 0; c < nv; ++c)
                s += V[(size_t)a * nv2 + (size_t)b * nv + c] * OVOV(&B, q, d, r, c);
              zv[(((size_t)a * nv + b) * no + p) * nv + d] -= s;
            }
        ORACLE_INNER_FOR
        for (int a = 0; a < nv; ++a)
          for (int l = 0; l < no; ++l) {
            double s = 0.0;
            for (int b = 0; b < nv; ++b)
              for (int c = 0; c < nv; ++c)
                s += V[(size_t)a * nv2 + (size_t)b * nv + c] * OVOV(&B, l, b, r, c);
            zo[(((size_t)a * no + q) * no + p) * no + l] += s;
          }
        fl += 2LL * nv * nv * nv * nv;
      }
    }
#pragma omp critical
    {
      for (size_t x = 0; x < nzv; ++x) Zv[x] += zv[x];
      for (size_t x = 0; x < nzo; ++x) Zo[x] += zo[x];
    }
    free(W); free(S); free(tau); free(V); free(zv); free(zo);
  }
  if (flops) *flops = fl;
  free(T);
  return used;
}

/* (pq|rs) = sum_J L[J][p][q] L[J][r][s] over the n = no+nv active orbitals
 * (occupied first). */
static double eri(const double *L, int naux, int n, int p, int q, int r, int s) {
  double v = 0.0;
  size_t n2 = (size_t)n * n;
  for (int J = 0; J < naux; ++J)
    v += L[J * n2 + (size_t)p * n + q] * L[J * n2 + (size_t)r * n + s];
  return v;
}

/* One block of integrals G[p][q][r][s] = (p0+p q0+q | r0+r s0+s) for
 * p < np, q < nq, r < nr, s < ns (orbital offsets p0.. into the n orbitals). */
static double *eri_block(const double *L, int naux, int n, int p0, int np, int q0, int nq,
                         int r0, int nr, int s0, int ns) {
  double *G = (double *)malloc(((size_t)np * nq * nr * ns + 1) * sizeof(double));
  if (!G) return NULL;
#pragma omp parallel for collapse(2) schedule(static)
  for (int p = 0; p < np; ++p)
    for (int q = 0; q < nq; ++q)
      for (int r = 0; r < nr; ++r)
        for (int t = 0; t < ns; ++t)
          G[(((size_t)p * nq + q) * nr + r) * ns + t] =
              eri(L, naux, n, p0 + p, q0 + q, r0 + r, s0 + t);
  return G;
}

/* R1-dressed blocks from the first-order T1 transformation
 * g^_{pqrs} = -[p in v] sum_l R^p_l g_{lqrs} + [q in o] sum_e R^e_q g_{pers}
 *             -[r in v] sum_l R^r_l g_{pqls} + [s in o] sum_e R^e_s g_{pqre}
 * (H = exp(-T1) H exp(T1), differentiated along T1 = R1):
 *   g^_{bdck} = -sum_l R^b_l (ld|ck) - sum_l R^c_l (bd|lk) + sum_e R^e_k (bd|ce)
 *   g^_{ljck} =  sum_d R^d_j (ld|ck) - sum_m R^c_m (lj|mk) + sum_d R^d_k (lj|cd)
 *   g^_{jlkc} =  sum_d R^d_l (jd|kc)        g^_{dbkc} = -sum_l R^d_l (lb|kc)
 *   g^_{jbkc} = 0                           F^_{kc} = sum_ld [2(kc|ld)-(kd|lc)] R^d_l
 * The integrals (pq|rs) = sum_J L^J_pq L^J_rs of the ovvo, vvoo, oooo, oovv and
 * ovov kinds are formed once as blocks; the vvvv integrals of the first line
 * are contracted through the Cholesky vectors instead:
 * sum_e R^e_k (bd|ce) = sum_J L^J_bd (sum_e L^J_ce R^e_k). */
static void dressed_blocks(int no, int nv, const double *L, int naux,
                           const double *R1, double *hvvvo, double *hoovo,
                           double *hooov, double *hvvov, double *hF) {
  int n = no + nv;
  size_t n2 = (size_t)n * n;
#define R(i, a) R1[(size_t)(i) * nv + (a)]
#define V(p) (no + (p))
  /* Govvo[l][d][c][k] = (ld|ck), Gvvoo[b][d][l][k] = (bd|lk),
   * Goooo[l][j][m][k] = (lj|mk), Goovv[l][j][c][d] = (lj|cd),
   * Govov[j][d][k][c] = (jd|kc) */
  double *Govvo = eri_block(L, naux, n, 0, no, no, nv, no, nv, 0, no);
  double *Gvvoo = eri_block(L, naux, n, no, nv, no, nv, 0, no, 0, no);
  double *Goooo = eri_block(L, naux, n, 0, no, 0, no, 0, no, 0, no);
  double *Goovv = eri_block(L, naux, n, 0, no, 0, no, no, nv, no, nv);
  double *Govov = eri_block(L, naux, n, 0, no, no, nv, 0, no, no, nv);
#define OVVO(l, d, c, k) Govvo[(((size_t)(l) * nv + (d)) * nv + (c)) * no + (k)]
#define VVOO(b, d, l, k) Gvvoo[(((size_t)(b) * nv + (d)) * no + (l)) * no + (k)]
#define OOOO(l, j, m, k) Goooo[(((size_t)(l) * no + (j)) * no + (m)) * no + (k)]
#define OOVV(l, j, c, d) Goovv[(((size_t)(l) * no + (j)) * nv + (c)) * nv + (d)]
#define GOVOV(j, d, k, c) Govov[(((size_t)(j) * nv + (d)) * no + (k)) * nv + (c)]
  double *M = (double *)calloc((size_t)naux * nv * no + 1, sizeof(double));
#pragma omp parallel for collapse(2) schedule(static)
  for (int J = 0; J < naux; ++J)
    for (int c = 0; c < nv; ++c)
      for (int k = 0; k < no; ++k) {
        double s = 0.0;
        for (int e = 0; e < nv; ++e)
          s += L[J * n2 + (size_t)V(c) * n + V(e)] * R(k, e);
        M[((size_t)J * nv + c) * no + k] = s;
      }
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < nv; ++b)
    for (int d = 0; d < nv; ++d)
      for (int c = 0; c < nv; ++c)
        for (int k = 0; k < no; ++k) {
          double s = 0.0;
          for (int l = 0; l < no; ++l)
            s -= R(l, b) * OVVO(l, d, c, k);
          for (int l = 0; l < no; ++l)
            s -= R(l, c) * VVOO(b, d, l, k);
          for (int J = 0; J < naux; ++J)
            s += L[J * n2 + (size_t)V(b) * n + V(d)] *
                 M[((size_t)J * nv + c) * no + k];
          hvvvo[(((size_t)b * nv + d) * nv + c) * no + k] = s;
        }
#pragma omp parallel for collapse(2) schedule(static)
  for (int l = 0; l < no; ++l)
    for (int j = 0; j < no; ++j)
      for (int c = 0; c < nv; ++c)
        for (int k = 0; k < no; ++k) {
          double s = 0.0;
          for (int d = 0; d < nv; ++d)
            s += R(j, d) * OVVO(l, d, c, k);
          for (int m = 0; m < no; ++m)
            s -= R(m, c) * OOOO(l, j, m, k);
          for (int d = 0; d < nv; ++d)
            s += R(k, d) * OOVV(l, j, c, d);
          hoovo[(((size_t)l * no + j) * nv + c) * no + k] = s;
        }
#pragma omp parallel for collapse(2) schedule(static)
  for (int j = 0; j < no; ++j)
    for (int l = 0; l < no; ++l)
      for (int k = 0; k < no; ++k)
        for (int c = 0; c < nv; ++c) {
          double s = 0.0;
          for (int d = 0; d < nv; ++d)
            s += R(l, d) * GOVOV(j, d, k, c);
          hooov[(((size_t)j * no + l) * no + k) * nv + c] = s;
        }
#pragma omp parallel for collapse(2) schedule(static)
  for (int d = 0; d < nv; ++d)
    for (int b = 0; b < nv; ++b)
      for (int k = 0; k < no; ++k)
        for (int c = 0; c < nv; ++c) {
          double s = 0.0;
          for (int l = 0; l < no; ++l)
            s -= R(l, d) * GOVOV(l, b, k, c);
          hvvov[(((size_t)d * nv + b) * no + k) * nv + c] = s;
        }
  for (int k = 0; k < no; ++k)
    for (int c = 0; c < nv; ++c) {
      double s = 0.0;
      for (int l = 0; l < no; ++l)
        for (int d = 0; d < nv; ++d)
          s += (2.0 * GOVOV(k, c, l, d) - GOVOV(k, d, l, c)) * R(l, d);
      hF[(size_t)k * nv + c] = s;
    }
  free(M);
  free(Govvo); free(Gvvoo); free(Goooo); free(Goovv); free(Govov);
#undef OVVO
#undef VVOO
#undef OOOO
#undef OOVV
#undef GOVOV
#undef R
#undef V
}

/* Right Jacobian transformation of nvec trial vectors (R1[n][i][a],
 * R2[n][i][j][a][b], frequency w[n]):
 *   W_R  = P[ sum_d R^{ad}_{ij} g_{bdck} - sum_l R^{ab}_{il} g_{ljck} ]
 *        + P[ sum_d t^{ad}_{ij} g^_{bdck} - sum_l t^{ab}_{il} g^_{ljck} ]
 *   R3   = W_R / (w - eps);  R~3 its contravariant form
 *   rho~ = contractions(R~3; g, F) + contractions(tau~3; g^, F^)
 *   rho2 = (1/3) P^{ab}_{ij}(2 rho~ + rho~^{ba});  rho1 = rho~1.
 * The integrals are symmetric (T1 = 0), given as the five blocks plus the
 * Cholesky vectors chol_L[naux][n][n] for the dressed blocks.
 * The tau~3 . g^ contractions are done directly here (Algorithm 2's
 * intermediates are the GPU library's way to the same sums).
 * Returns threads used. */
int oracle_jacobian(int no, int nv, const double *eps_o, const double *eps_v,
                    const double *t2, const double *vvvo, const double *oovo,
                    const double *ooov, const double *ovov, const double *vvov,
                    const double *F_ov, const double *chol_L, int naux,
                    int nvec, const double *w, const double *R1,
                    const double *R2, int ntri, const int *tri, double *rho1,
                    double *rho2, long long *flops, int nthreads) {
  size_t nv3 = (size_t)nv * nv * nv, n1 = (size_t)no * nv,
         n2 = (size_t)no * no * nv * nv;
  size_t nvvvo = nv3 * no, noovo = (size_t)no * no * nv * no,
         nooov = (size_t)no * no * no * nv, nvvov = nv3 * no;
  int *T = NULL;
  int nt = list_triples(no, ntri, tri, &T);
  if (nt < 0) return -1;
  int used = set_threads(nthreads);
  long long fl_total = 0;
  for (int vec = 0; vec < nvec; ++vec) {
    const double *r1 = R1 + vec * n1, *r2 = R2 + vec * n2;
    double *hvvvo = (double *)malloc(nvvvo * sizeof(double));
    double *hoovo = (double *)malloc(noovo * sizeof(double) + 8);
    double *hooov = (double *)malloc(nooov * sizeof(double) + 8);
    double *hvvov = (double *)malloc(nvvov * sizeof(double));
    double *hF = (double *)malloc(n1 * sizeof(double) + 8);
    double *zero_ovov = (double *)calloc(n2 + 1, sizeof(double));
    dressed_blocks(no, nv, chol_L, naux, r1, hvvvo, hoovo, hooov, hvvov, hF);
    blocks_t Bg = {no, nv, eps_o, eps_v, t2, vvvo, oovo, ooov, ovov, vvov, F_ov};
    blocks_t Bh = {no, nv, eps_o, eps_v, t2, hvvvo, hoovo, hooov, zero_ovov,
                   hvvov, hF};
    double *om1 = (double *)calloc(n1 + 1, sizeof(double));
    double *omt = (double *)calloc(n2 + 1, sizeof(double));
    long long fl = 0;
#pragma omp parallel if (nt >= used) reduction(+ : fl)
    {
      double *W = (double *)malloc(nv3 * sizeof(double));
      double *W2 = (double *)malloc(nv3 * sizeof(double));
      double *S = (double *)malloc(nv3 * sizeof(double));
      double *tau = (double *)malloc(nv3 * sizeof(double));
      double *V = (double *)malloc(nv3 * sizeof(double));
      double *m1 = (double *)calloc(n1 + 1, sizeof(double));
      double *mt = (double *)calloc(n2 + 1, sizeof(double));
#pragma omp for schedule(dynamic, 1)
      for (int t = 0; t < nt; ++t) {
        const int *ijk = T + 3 * t;
        int maps[6][3];
        int np = distinct_perms(ijk, maps);
        if (np == 0) continue;
        /* R3 and its contractions with the undressed integrals */
        build_W(no, nv, r2, vvvo, oovo, ijk, W, S, &fl);
        build_W(no, nv, t2, hvvvo, hoovo, ijk, W2, S, &fl);
        for (size_t x = 0; x < nv3; ++x) W[x] += W2[x];
        divide_denominator(&Bg, ijk, w[vec], W, tau);
        contravariant(nv, tau, S);
        for (int u = 0; u < np; ++u) {
          permuted_view(nv, S, maps[u], V);
          contract_omega(&Bg, V, ijk[maps[u][0]], ijk[maps[u][1]],
                         ijk[maps[u][2]], m1, mt, &fl);
        }
        /* tau3 and its contractions with the dressed integrals */
        build_W(no, nv, t2, vvvo, oovo, ijk, W, S, &fl);
        divide_denominator(&Bg, ijk, 0.0, W, tau);
        contravariant(nv, tau, S);
        for (int u = 0; u < np; ++u) {
          permuted_view(nv, S, maps[u], V);
          contract_omega(&Bh, V, ijk[maps[u][0]], ijk[maps[u][1]],
                         ijk[maps[u][2]], m1, mt, &fl);
        }
      }
#pragma omp critical
      {
        for (size_t x = 0; x < n1; ++x) om1[x] += m1[x];
        for (size_t x = 0; x < n2; ++x) omt[x] += mt[x];
      }
      free(W); free(W2); free(S); free(tau); free(V); free(m1); free(mt);
    }
    memcpy(rho1 + vec * n1, om1, n1 * sizeof(double));
    back_transform(no, nv, omt, rho2 + vec * n2);
    fl_total += fl;
    free(om1); free(omt); free(hvvvo); free(hoovo); free(hooov); free(hvvov);
    free(hF); free(zero_ovov);
  }
  if (flops) *flops = fl_total;
  free(T);
  return used;
}

/* ------------------------------------------------------------------------
 * Left (transpose) Jacobian transformation, triples part.
 *
 * The paper's transpose-Jacobian paragraph (section "Implementation") builds
 * the covariant L3 amplitudes with contractions like those of tau3 plus outer
 * products, takes their contravariant form by eq. "contra_t", and contracts
 * them back, after a separate loop that contracts tau3; Algorithm 3 gives the
 * same L3 amplitudes (an outer product of L1 with g_ovov, one of L2 with F,
 * and two contractions of L2 with integrals, permuted by P and divided by
 * (w - eps)).  Here the left transformation is read as the exact transpose of the right
 * one (oracle_jacobian) under the plain inner product over the elements of
 * (R1, R2): sigma = J(w)^T L, so that sum L.rho(R) = sum sigma(L).R for every
 * pair-symmetric R2.  With Lt2 = the back-transform applied to L2 (the
 * back-transform (1/3) P^{ab}_{ij}(2X + X^{ba}) is its own transpose) that
 * gives, per ordered triple (p,q,r) (a distinct permutation of a loop triple,
 * V the contravariant amplitudes viewed with x, y, z in the slots of p, q, r):
 *
 *   X_pqr[x][y][z] = L1[p][x] g_{qyrz} + Lt2[p][q][x][y] F[r][z]
 *                  + sum_d Lt2[p][q][x][d] g_{dyrz} - sum_l Lt2[p][l][x][y] g_{qlrz}
 *   L3 = (w - eps)^{-1} P X,  V = contravariant(L3)
 *   sigma2[p][q][x][d] += sum_yz V g_{ydzr}      sigma2[p][l][x][y] -= sum_z V g_{lqzr}
 *   G[y][d][z][r]      += sum_x V t[p][q][x][d]  H[l][q][z][r]      += sum_xy V t[p][l][x][y]
 *
 * and, from the tau3 loop (V = contravariant tau3),
 *   Q[r][z] += sum_xy Lt2[p][q][x][y] V[x][y][z]
 *   sigma1[l][d] -= sum_xyz Lt2[p][l][x][y] V[x][y][z] (qd|rz)
 *                 + sum_xyz Lt2[p][q][x][d] V[x][y][z] (ly|rz)
 * (the transposes of the tau~3 . g^_ooov and tau~3 . g^_vvov terms).  After
 * the loops the R1 dependence of the dressed integrals is transposed:
 *   sigma1 += F^(Q) (F^_kc = sum_ld [2(kc|ld) - (kd|lc)] x_ld is symmetric)
 *   sigma1[l][b] -= sum G[b][d][c][k] (ld|ck)   sigma1[l][c] -= sum G[b][d][c][k] (bd|lk)
 *   sigma1[k][e] += sum G[b][d][c][k] (bd|ce)   (vvvv through the Cholesky vectors)
 *   sigma1[j][d] -= sum H[l][j][c][k] (ld|ck)   sigma1[m][c] += sum H[l][j][c][k] (lj|mk)
 *   sigma1[k][d] -= sum H[l][j][c][k] (lj|cd)
 *   sigma2 <- (sigma2 + sigma2^{T pair}) / 2.
 * Cost: 8 nv^4 per distinct permutation (tau3, X, sigma2 and G, 2 nv^4 each).
 * Symmetric integrals (T1 = 0), as oracle_jacobian.
 * ---------------------------------------------------------------------- */

/* X_pqr of the L3 amplitudes (see above); lt2 = the back-transformed L2 */
static void build_X(const blocks_t *B, const double *l1, const double *lt2, int p, int q,
                    int r, double *Xout, long long *flops) {
  int no = B->no, nv = B->nv;
  size_t nv2 = (size_t)nv * nv;
  ORACLE_INNER_FOR
  for (int x = 0; x < nv; ++x)
    for (int y = 0; y < nv; ++y) {
      double *row = Xout + (size_t)x * nv2 + (size_t)y * nv;
      const double l1x = l1[(size_t)p * nv + x];
      const double lxy = lt2[(((size_t)p * no + q) * nv + x) * nv + y];
      for (int z = 0; z < nv; ++z)
        row[z] = l1x * OVOV(B, q, y, r, z) + lxy * B->F_ov[(size_t)r * nv + z];
      for (int d = 0; d < nv; ++d) {
        const double ld = lt2[(((size_t)p * no + q) * nv + x) * nv + d];
        for (int z = 0; z < nv; ++z) row[z] += ld * VVOV(B, d, y, r, z);
      }
      for (int l = 0; l < no; ++l) {
        const double ll = lt2[(((size_t)p * no + l) * nv + x) * nv + y];
        for (int z = 0; z < nv; ++z) row[z] -= ll * OOOV(B, q, l, r, z);
      }
    }
  if (flops) *flops += 2LL * nv * nv * nv * nv;
}

/* L3 numerator P X for one unique triple (placement as in build_W) */
static void build_PX(const blocks_t *B, const double *l1, const double *lt2, const int ijk[3],
                     double *W, double *Xs, long long *flops) {
  int nv = B->nv;
  size_t nv2 = (size_t)nv * nv, nv3 = nv2 * nv;
  memset(W, 0, nv3 * sizeof(double));
  int done[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < 6; ++s) {
    if (done[s]) continue;
    int p = ijk[PERM6[s][0]], q = ijk[PERM6[s][1]], r = ijk[PERM6[s][2]];
    build_X(B, l1, lt2, p, q, r, Xs, flops);
    for (int s2 = s; s2 < 6; ++s2) {
      if (ijk[PERM6[s2][0]] != p || ijk[PERM6[s2][1]] != q || ijk[PERM6[s2][2]] != r) continue;
      done[s2] = 1;
      const int *m = PERM6[s2];
      ORACLE_INNER_FOR
      for (int v0 = 0; v0 < nv; ++v0) {
        int v[3];
        v[0] = v0;
        for (v[1] = 0; v[1] < nv; ++v[1])
          for (v[2] = 0; v[2] < nv; ++v[2]) {
            size_t src = (size_t)v[m[0]] * nv2 + (size_t)v[m[1]] * nv + v[m[2]];
            W[(size_t)v[0] * nv2 + (size_t)v[1] * nv + v[2]] += Xs[src];
          }
      }
    }
  }
}

int oracle_left_jacobian(int no, int nv, const double *eps_o, const double *eps_v,
                         const double *t2, const double *vvvo, const double *oovo,
                         const double *ooov, const double *ovov, const double *vvov,
                         const double *F_ov, const double *chol_L, int naux, int nvec,
                         const double *w, const double *L1, const double *L2, int ntri,
                         const int *tri, double *sig1, double *sig2, long long *flops,
                         int nthreads) {
  size_t nv2 = (size_t)nv * nv, nv3 = nv2 * nv, n1 = (size_t)no * nv,
         n2 = (size_t)no * no * nv * nv;
  int n = no + nv;
  size_t nn = (size_t)n * n;
  int *T = NULL;
  int nt = list_triples(no, ntri, tri, &T);
  if (nt < 0) return -1;
  int used = set_threads(nthreads);
  blocks_t B = {no, nv, eps_o, eps_v, t2, vvvo, oovo, ooov, ovov, vvov, F_ov};
  long long fl_total = 0;
  for (int vec = 0; vec < nvec; ++vec) {
    const double *l1 = L1 + vec * n1, *l2 = L2 + vec * n2;
    double *lt2 = (double *)malloc(n2 * sizeof(double) + 8);
    back_transform(no, nv, l2, lt2);  /* the back-transform is its own transpose */
    double *s1 = (double *)calloc(n1 + 1, sizeof(double));
    double *s2 = (double *)calloc(n2 + 1, sizeof(double));
    double *Q = (double *)calloc(n1 + 1, sizeof(double));
    double *G = (double *)calloc(nv3 * no + 1, sizeof(double));
    double *H = (double *)calloc((size_t)no * no * nv * no + 1, sizeof(double));
    long long fl = 0;
    /* loop 1: tau3 and its contractions with Lt2 */
#pragma omp parallel if (nt >= used) reduction(+ : fl)
    {
      double *W = (double *)malloc(nv3 * sizeof(double));
      double *S = (double *)malloc(nv3 * sizeof(double));
      double *tau = (double *)malloc(nv3 * sizeof(double));
      double *V = (double *)malloc(nv3 * sizeof(double));
      double *q1 = (double *)calloc(n1 + 1, sizeof(double));
      double *m1 = (double *)calloc(n1 + 1, sizeof(double));
#pragma omp for schedule(dynamic, 1)
      for (int t = 0; t < nt; ++t) {
        const int *ijk = T + 3 * t;
        int maps[6][3];
        int np = distinct_perms(ijk, maps);
        if (np == 0) continue;
        build_W(no, nv, t2, vvvo, oovo, ijk, W, S, &fl);
        divide_denominator(&B, ijk, 0.0, W, tau);
        contravariant(nv, tau, S);
        for (int u = 0; u < np; ++u) {
          int p = ijk[maps[u][0]], q = ijk[maps[u][1]], r = ijk[maps[u][2]];
          permuted_view(nv, S, maps[u], V);
          for (int x = 0; x < nv; ++x)
            for (int y = 0; y < nv; ++y) {
              const double lq = lt2[(((size_t)p * no + q) * nv + x) * nv + y];
              const double *vr = V + (size_t)x * nv2 + (size_t)y * nv;
              for (int z = 0; z < nv; ++z) q1[(size_t)r * nv + z] += lq * vr[z];
            }
          /* - sum Lt2[p][l][x][y] V[x][y][z] (qd|rz) */
          for (int x = 0; x < nv; ++x)
            for (int y = 0; y < nv; ++y) {
              const double *vr = V + (size_t)x * nv2 + (size_t)y * nv;
              for (int d = 0; d < nv; ++d) {
                double s = 0.0;
                for (int z = 0; z < nv; ++z) s += vr[z] * OVOV(&B, q, d, r, z);
                for (int l = 0; l < no; ++l)
                  m1[(size_t)l * nv + d] -= lt2[(((size_t)p * no + l) * nv + x) * nv + y] * s;
              }
            }
          /* - sum Lt2[p][q][x][d] V[x][y][z] (ly|rz) */
          for (int x = 0; x < nv; ++x)
            for (int l = 0; l < no; ++l) {
              double s = 0.0;
              for (int y = 0; y < nv; ++y)
                for (int z = 0; z < nv; ++z)
                  s += V[(size_t)x * nv2 + (size_t)y * nv + z] * OVOV(&B, l, y, r, z);
              for (int d = 0; d < nv; ++d)
                m1[(size_t)l * nv + d] -= lt2[(((size_t)p * no + q) * nv + x) * nv + d] * s;
            }
        }
      }
#pragma omp critical
      {
        for (size_t x = 0; x < n1; ++x) Q[x] += q1[x];
        for (size_t x = 0; x < n1; ++x) s1[x] += m1[x];
      }
      free(W); free(S); free(tau); free(V); free(q1); free(m1);
    }
    /* loop 2: L3, its contravariant form and its contractions */
#pragma omp parallel if (nt >= used) reduction(+ : fl)
    {
      double *W = (double *)malloc(nv3 * sizeof(double));
      double *S = (double *)malloc(nv3 * sizeof(double));
      double *l3 = (double *)malloc(nv3 * sizeof(double));
      double *V = (double *)malloc(nv3 * sizeof(double));
      double *m2 = (double *)calloc(n2 + 1, sizeof(double));
      double *g = (double *)calloc(nv3 * no + 1, sizeof(double));
      double *h = (double *)calloc((size_t)no * no * nv * no + 1, sizeof(double));
#pragma omp for schedule(dynamic, 1)
      for (int t = 0; t < nt; ++t) {
        const int *ijk = T + 3 * t;
        int maps[6][3];
        int np = distinct_perms(ijk, maps);
        if (np == 0) continue;
        build_PX(&B, l1, lt2, ijk, W, S, &fl);
        divide_denominator(&B, ijk, w[vec], W, l3);
        contravariant(nv, l3, S);
        for (int u = 0; u < np; ++u) {
          int p = ijk[maps[u][0]], q = ijk[maps[u][1]], r = ijk[maps[u][2]];
          permuted_view(nv, S, maps[u], V);
          ORACLE_INNER_FOR
          for (int x = 0; x < nv; ++x) {
            for (int d = 0; d < nv; ++d) {  /* sigma2[p][q][x][d] += sum_yz V g_{ydzr} */
              double s = 0.0;
              for (int y = 0; y < nv; ++y)
                for (int z = 0; z < nv; ++z)
                  s += V[(size_t)x * nv2 + (size_t)y * nv + z] * VVVO(&B, y, d, z, r);
              m2[(((size_t)p * no + q) * nv + x) * nv + d] += s;
            }
            for (int y = 0; y < nv; ++y)    /* sigma2[p][l][x][y] -= sum_z V g_{lqzr} */
              for (int l = 0; l < no; ++l) {
                double s = 0.0;
                for (int z = 0; z < nv; ++z)
                  s += V[(size_t)x * nv2 + (size_t)y * nv + z] * OOVO(&B, l, q, z, r);
                m2[(((size_t)p * no + l) * nv + x) * nv + y] -= s;
              }
          }
          ORACLE_INNER_FOR
          for (int y = 0; y < nv; ++y)      /* G[y][d][z][r] += sum_x V t[p][q][x][d] */
            for (int d = 0; d < nv; ++d)
              for (int z = 0; z < nv; ++z) {
                double s = 0.0;
                for (int x = 0; x < nv; ++x)
                  s += V[(size_t)x * nv2 + (size_t)y * nv + z] * T2(&B, p, q, x, d);
                g[(((size_t)y * nv + d) * nv + z) * no + r] += s;
              }
          for (int z = 0; z < nv; ++z)      /* H[l][q][z][r] += sum_xy V t[p][l][x][y] */
            for (int l = 0; l < no; ++l) {
              double s = 0.0;
              for (int x = 0; x < nv; ++x)
                for (int y = 0; y < nv; ++y)
                  s += V[(size_t)x * nv2 + (size_t)y * nv + z] * T2(&B, p, l, x, y);
              h[(((size_t)l * no + q) * nv + z) * no + r] += s;
            }
          fl += 4LL * nv * nv * nv * nv;
        }
      }
#pragma omp critical
      {
        for (size_t x = 0; x < n2; ++x) s2[x] += m2[x];
        for (size_t x = 0; x < nv3 * no; ++x) G[x] += g[x];
        for (size_t x = 0; x < (size_t)no * no * nv * no; ++x) H[x] += h[x];
      }
      free(W); free(S); free(l3); free(V); free(m2); free(g); free(h);
    }
    /* the R1 dependence of F^ and of the dressed integrals, transposed */
    const double *L = chol_L;
#define V_(p) (no + (p))
    for (int l = 0; l < no; ++l)
      for (int d = 0; d < nv; ++d) {
        double s = 0.0;
        for (int k = 0; k < no; ++k)
          for (int c = 0; c < nv; ++c)
            s += Q[(size_t)k * nv + c] * (2.0 * OVOV(&B, k, c, l, d) - OVOV(&B, k, d, l, c));
        s1[(size_t)l * nv + d] += s;
      }
#pragma omp parallel for schedule(static)
    for (int l = 0; l < no; ++l) {
      for (int b = 0; b < nv; ++b) {   /* - sum G[b][d][c][k] (ld|ck) */
        double s = 0.0;
        for (int d = 0; d < nv; ++d)
          for (int c = 0; c < nv; ++c)
            for (int k = 0; k < no; ++k)
              s += G[(((size_t)b * nv + d) * nv + c) * no + k] * eri(L, naux, n, l, V_(d), V_(c), k);
        s1[(size_t)l * nv + b] -= s;
      }
      for (int c = 0; c < nv; ++c) {   /* - sum G[b][d][c][k] (bd|lk) */
        double s = 0.0;
        for (int b = 0; b < nv; ++b)
          for (int d = 0; d < nv; ++d)
            for (int k = 0; k < no; ++k)
              s += G[(((size_t)b * nv + d) * nv + c) * no + k] * eri(L, naux, n, V_(b), V_(d), l, k);
        s1[(size_t)l * nv + c] -= s;
      }
    }
    { /* + sum G[b][d][c][k] (bd|ce) = sum_J (sum_bd G L^J_bd) L^J_ce */
      double *N = (double *)calloc((size_t)naux * nv * no + 1, sizeof(double));
#pragma omp parallel for schedule(static)
      for (int J = 0; J < naux; ++J)
        for (int c = 0; c < nv; ++c)
          for (int k = 0; k < no; ++k) {
            double s = 0.0;
            for (int b = 0; b < nv; ++b)
              for (int d = 0; d < nv; ++d)
                s += L[J * nn + (size_t)V_(b) * n + V_(d)] * G[(((size_t)b * nv + d) * nv + c) * no + k];
            N[((size_t)J * nv + c) * no + k] = s;
          }
      for (int k = 0; k < no; ++k)
        for (int e = 0; e < nv; ++e) {
          double s = 0.0;
          for (int J = 0; J < naux; ++J)
            for (int c = 0; c < nv; ++c)
              s += N[((size_t)J * nv + c) * no + k] * L[J * nn + (size_t)V_(c) * n + V_(e)];
          s1[(size_t)k * nv + e] += s;
        }
      free(N);
    }
#define HH(l, j, c, k) H[(((size_t)(l) * no + (j)) * nv + (c)) * no + (k)]
    for (int j = 0; j < no; ++j)       /* - sum H[l][j][c][k] (ld|ck) */
      for (int d = 0; d < nv; ++d) {
        double s = 0.0;
        for (int l = 0; l < no; ++l)
          for (int c = 0; c < nv; ++c)
            for (int k = 0; k < no; ++k) s += HH(l, j, c, k) * eri(L, naux, n, l, V_(d), V_(c), k);
        s1[(size_t)j * nv + d] -= s;
      }
    for (int m = 0; m < no; ++m)       /* + sum H[l][j][c][k] (lj|mk) */
      for (int c = 0; c < nv; ++c) {
        double s = 0.0;
        for (int l = 0; l < no; ++l)
          for (int j = 0; j < no; ++j)
            for (int k = 0; k < no; ++k) s += HH(l, j, c, k) * eri(L, naux, n, l, j, m, k);
        s1[(size_t)m * nv + c] += s;
      }
    for (int k = 0; k < no; ++k)       /* - sum H[l][j][c][k] (lj|cd) */
      for (int d = 0; d < nv; ++d) {
        double s = 0.0;
        for (int l = 0; l < no; ++l)
          for (int j = 0; j < no; ++j)
            for (int c = 0; c < nv; ++c) s += HH(l, j, c, k) * eri(L, naux, n, l, j, V_(c), V_(d));
        s1[(size_t)k * nv + d] -= s;
      }
#undef HH
#undef V_
    memcpy(sig1 + vec * n1, s1, n1 * sizeof(double));
    for (int i = 0; i < no; ++i)
      for (int j = 0; j < no; ++j)
        for (int a = 0; a < nv; ++a)
          for (int b = 0; b < nv; ++b)
            sig2[vec * n2 + (((size_t)i * no + j) * nv + a) * nv + b] =
                0.5 * (s2[(((size_t)i * no + j) * nv + a) * nv + b] +
                       s2[(((size_t)j * no + i) * nv + b) * nv + a]);
    fl_total += fl;
    free(lt2); free(s1); free(s2); free(Q); free(G); free(H);
  }
  if (flops) *flops = fl_total;
  free(T);
  return used;
}

/* ------------------------------------------------------------------------
 * Algorithm 3: the triples contributions to the one-electron density
 * D^{m,0}_{pq} = <m|E_pq|CC> of a left state (L1, L2) at frequency w; with
 * w = 0 and the ground-state multipliers in place of (L1, L2) the same steps
 * give D^{0,0} (the paragraph after Algorithm 3).
 *
 * The L3 amplitudes are the covariant triples of the left state exactly as
 * the left transformation above builds them: X from L1 and Lt2 (the
 * back-transformed L2), L3 = P X / (w - eps), L~3 = contravariant(L3).  The
 * doubles of the left state enter the ov block through Lt2 as well: that
 * term is the derivative of sum L.Omega with respect to F_kc.
 *
 * Occupied loop, triples i >= j >= k, every distinct permutation (p,q,r) of a
 * triple (V_X = the view of X_{ijk} with the virtual slots permuted alike):
 *   tau = W / (0 - eps) (Algorithm 1),  tau~ = contravariant(tau)
 *   Y[c][l][p][r] += sum_ab V_L~[a][b][c] t[l][q][a][b]
 *   Dvv[c][d]     += 1/2 sum_ab V_L~[a][b][c] V_tau[a][b][d]
 *   Dov[r][c]     += sum_ab Lt2[p][q][a][b] V_tau~[a][b][c]
 * after it  Dov[l][d] -= sum_cik Y[c][l][i][k] t[k][i][c][d].
 * Virtual loop, a >= b >= c, every distinct ordering (x,y,z) of the virtual
 * triple and every ordered occupied triple (i,j,k): tau^{xyz}_{ijk} and
 * L3^{xyz}_{ijk} from the same formulas, and
 *   Doo[l][k]     -= 1/2 sum_ij L~^{xyz}_{ijk} tau^{xyz}_{ijl}.
 * The vo block has no triples term.  tau and L3 take the formula's values at
 * every index (also i = j = k and a = b = c), as the two loops build them.
 * Cost: 6 nv^4 per distinct permutation (tau3, X, Dvv) plus 4 nv^4 no^3 for
 * the virtual loop (tau3 and X again): 10 nv^4 no^3 in all.
 * ---------------------------------------------------------------------- */

/* B^{xyz}_{pqr} and X^{xyz}_{pqr} of one element (the tau3 bracket and the L3
 * numerator of one ordered triple pair) */
static double elem_B(const blocks_t *B, int x, int y, int z, int p, int q, int r) {
  int no = B->no, nv = B->nv;
  double s = 0.0;
  for (int d = 0; d < nv; ++d) s += T2(B, p, q, x, d) * VVVO(B, y, d, z, r);
  for (int l = 0; l < no; ++l) s -= T2(B, p, l, x, y) * OOVO(B, l, q, z, r);
  return s;
}

static double elem_X(const blocks_t *B, const double *l1, const double *lt2, int x, int y,
                     int z, int p, int q, int r) {
  int no = B->no, nv = B->nv;
#define LT(i, j, a, b) lt2[(((size_t)(i) * no + (j)) * nv + (a)) * nv + (b)]
  double s = l1[(size_t)p * nv + x] * OVOV(B, q, y, r, z) + LT(p, q, x, y) * B->F_ov[(size_t)r * nv + z];
  for (int d = 0; d < nv; ++d) s += LT(p, q, x, d) * VVOV(B, d, y, r, z);
  for (int l = 0; l < no; ++l) s -= LT(p, l, x, y) * OOOV(B, q, l, r, z);
#undef LT
  return s;
}

/* index in PERM6 of the slot map m */
static int perm_index(const int m[3]) {
  for (int s = 0; s < 6; ++s)
    if (PERM6[s][0] == m[0] && PERM6[s][1] == m[1] && PERM6[s][2] == m[2]) return s;
  return -1;
}

int oracle_density(int no, int nv, const double *eps_o, const double *eps_v,
                   const double *t2, const double *vvvo, const double *oovo,
                   const double *ooov, const double *ovov, const double *vvov,
                   const double *F_ov, double w, const double *L1, const double *L2,
                   double *Doo, double *Dov, double *Dvv, long long *flops, int nthreads) {
  size_t nv2 = (size_t)nv * nv, nv3 = nv2 * nv, n1 = (size_t)no * nv,
         n2 = (size_t)no * no * nv * nv, no3 = (size_t)no * no * no;
  size_t ny = (size_t)nv * no * no * no;
  int *T = NULL;
  int nt = list_triples(no, 0, NULL, &T);
  if (nt < 0) return -1;
  int used = set_threads(nthreads);
  blocks_t B = {no, nv, eps_o, eps_v, t2, vvvo, oovo, ooov, ovov, vvov, F_ov};
  double *lt2 = (double *)malloc(n2 * sizeof(double) + 8);
  back_transform(no, nv, L2, lt2);
  double *Y = (double *)calloc(ny + 1, sizeof(double));
  double *dvv = (double *)calloc(nv2 + 1, sizeof(double));
  double *dov = (double *)calloc(n1 + 1, sizeof(double));
  double *doo = (double *)calloc((size_t)no * no + 1, sizeof(double));
  long long fl = 0;
  /* occupied loop */
#pragma omp parallel if (nt >= used) reduction(+ : fl)
  {
    double *W = (double *)malloc(nv3 * sizeof(double) + 8);
    double *S = (double *)malloc(nv3 * sizeof(double) + 8);
    double *tau = (double *)malloc(nv3 * sizeof(double) + 8);
    double *tt = (double *)malloc(nv3 * sizeof(double) + 8);
    double *l3 = (double *)malloc(nv3 * sizeof(double) + 8);
    double *lt = (double *)malloc(nv3 * sizeof(double) + 8);
    double *VL = (double *)malloc(nv3 * sizeof(double) + 8);
    double *Vt = (double *)malloc(nv3 * sizeof(double) + 8);
    double *Vtt = (double *)malloc(nv3 * sizeof(double) + 8);
    double *y = (double *)calloc(ny + 1, sizeof(double));
    double *mvv = (double *)calloc(nv2 + 1, sizeof(double));
    double *mov = (double *)calloc(n1 + 1, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < nt; ++t) {
      const int *ijk = T + 3 * t;
      int maps[6][3];
      int np = distinct_perms(ijk, maps);
      if (np == 0) continue;
      build_W(no, nv, t2, vvvo, oovo, ijk, W, S, &fl);
      divide_denominator(&B, ijk, 0.0, W, tau);
      contravariant(nv, tau, tt);
      build_PX(&B, L1, lt2, ijk, W, S, &fl);
      divide_denominator(&B, ijk, w, W, l3);
      contravariant(nv, l3, lt);
      for (int u = 0; u < np; ++u) {
        int p = ijk[maps[u][0]], q = ijk[maps[u][1]], r = ijk[maps[u][2]];
        permuted_view(nv, lt, maps[u], VL);
        permuted_view(nv, tau, maps[u], Vt);
        permuted_view(nv, tt, maps[u], Vtt);
        ORACLE_INNER_FOR
        for (int c = 0; c < nv; ++c) {
          for (int l = 0; l < no; ++l) {   /* Y[c][l][p][r] */
            double s = 0.0;
            for (int a = 0; a < nv; ++a)
              for (int b = 0; b < nv; ++b)
                s += VL[(size_t)a * nv2 + (size_t)b * nv + c] * T2(&B, l, q, a, b);
            y[(((size_t)c * no + l) * no + p) * no + r] += s;
          }
          for (int d = 0; d < nv; ++d) {   /* Dvv[c][d] */
            double s = 0.0;
            for (int a = 0; a < nv; ++a)
              for (int b = 0; b < nv; ++b)
                s += VL[(size_t)a * nv2 + (size_t)b * nv + c] * Vt[(size_t)a * nv2 + (size_t)b * nv + d];
            mvv[(size_t)c * nv + d] += 0.5 * s;
          }
          double s = 0.0;                  /* Dov[r][c] */
          for (int a = 0; a < nv; ++a)
            for (int b = 0; b < nv; ++b)
              s += lt2[(((size_t)p * no + q) * nv + a) * nv + b] * Vtt[(size_t)a * nv2 + (size_t)b * nv + c];
          mov[(size_t)r * nv + c] += s;
        }
        fl += 2LL * nv * nv * nv * nv;
      }
    }
#pragma omp critical
    {
      for (size_t x = 0; x < ny; ++x) Y[x] += y[x];
      for (size_t x = 0; x < nv2; ++x) dvv[x] += mvv[x];
      for (size_t x = 0; x < n1; ++x) dov[x] += mov[x];
    }
    free(W); free(S); free(tau); free(tt); free(l3); free(lt); free(VL); free(Vt); free(Vtt);
    free(y); free(mvv); free(mov);
  }
  /* Dov[l][d] -= sum_{c,i,k} Y[c][l][i][k] t[k][i][c][d] */
  for (int l = 0; l < no; ++l)
    for (int d = 0; d < nv; ++d) {
      double s = 0.0;
      for (int c = 0; c < nv; ++c)
        for (int i = 0; i < no; ++i)
          for (int k = 0; k < no; ++k)
            s += Y[(((size_t)c * no + l) * no + i) * no + k] * T2(&B, k, i, c, d);
      dov[(size_t)l * nv + d] -= s;
    }
  /* virtual loop over a >= b >= c */
  int nvt = 0;
  int *V3 = (int *)malloc(sizeof(int) * 3 * ((size_t)nv * nv * nv + 1));
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b <= a; ++b)
      for (int c = 0; c <= b; ++c) {
        if (a == b && b == c) continue;
        V3[3 * nvt] = a;
        V3[3 * nvt + 1] = b;
        V3[3 * nvt + 2] = c;
        ++nvt;
      }
  /* the composed slot maps pi o m and the contravariant partners, as PERM6
   * indices */
  int comp[6][6];
  for (int s = 0; s < 6; ++s)
    for (int u = 0; u < 6; ++u) {
      int m[3] = {PERM6[s][PERM6[u][0]], PERM6[s][PERM6[u][1]], PERM6[s][PERM6[u][2]]};
      comp[s][u] = perm_index(m);
    }
  /* contravariant partners: orderings (x,z,y), (z,y,x), (y,x,z), (y,z,x),
   * (z,x,y) of an ordering (x,y,z), i.e. the slot maps PERM6[3], [2], [1],
   * [4], [5] composed after it */
#pragma omp parallel reduction(+ : fl)
  {
    double *Bt = (double *)malloc(6 * no3 * sizeof(double) + 8);
    double *Bx = (double *)malloc(6 * no3 * sizeof(double) + 8);
    double *tv = (double *)malloc(6 * no3 * sizeof(double) + 8);
    double *lv = (double *)malloc(6 * no3 * sizeof(double) + 8);
    double *ltv = (double *)malloc(no3 * sizeof(double) + 8);
    double *moo = (double *)calloc((size_t)no * no + 1, sizeof(double));
#pragma omp for schedule(dynamic, 4)
    for (int t = 0; t < nvt; ++t) {
      const int *v = V3 + 3 * t;
      for (int s = 0; s < 6; ++s) {
        int x = v[PERM6[s][0]], yy = v[PERM6[s][1]], z = v[PERM6[s][2]];
        for (int p = 0; p < no; ++p)
          for (int q = 0; q < no; ++q)
            for (int r = 0; r < no; ++r) {
              size_t o = ((size_t)p * no + q) * no + r;
              Bt[s * no3 + o] = elem_B(&B, x, yy, z, p, q, r);
              Bx[s * no3 + o] = elem_X(&B, L1, lt2, x, yy, z, p, q, r);
            }
        fl += 4LL * nv * (long long)no3;
      }
      /* tau and L3 at every ordering pi: P sums term u = B^{ordering pi o m_u}
       * at the occupied triple (o_{m0}, o_{m1}, o_{m2}), m_u = PERM6[u] */
      const double e = eps_v[v[0]] + eps_v[v[1]] + eps_v[v[2]];
      for (int s = 0; s < 6; ++s)
        for (int i = 0; i < no; ++i)
          for (int j = 0; j < no; ++j)
            for (int k = 0; k < no; ++k) {
              const int o[3] = {i, j, k};
              double wt = 0.0, wx = 0.0;
              for (int u = 0; u < 6; ++u) {
                size_t src = ((size_t)o[PERM6[u][0]] * no + o[PERM6[u][1]]) * no + o[PERM6[u][2]];
                wt += Bt[comp[s][u] * no3 + src];
                wx += Bx[comp[s][u] * no3 + src];
              }
              const double den = e - eps_o[i] - eps_o[j] - eps_o[k];
              size_t x = ((size_t)i * no + j) * no + k;
              tv[s * no3 + x] = wt / (0.0 - den);
              lv[s * no3 + x] = wx / (w - den);
            }
      int maps[6][3];
      int nd = distinct_perms(v, maps);
      for (int u = 0; u < nd; ++u) {
        const int s = perm_index(maps[u]);
        /* L~ at ordering s: 4 L^{xyz} - 2 L^{xzy} - 2 L^{zyx} - 2 L^{yxz}
         * + L^{yzx} + L^{zxy} */
        for (size_t x = 0; x < no3; ++x)
          ltv[x] = 4.0 * lv[s * no3 + x] - 2.0 * lv[comp[s][3] * no3 + x] -
                   2.0 * lv[comp[s][2] * no3 + x] - 2.0 * lv[comp[s][1] * no3 + x] +
                   lv[comp[s][4] * no3 + x] + lv[comp[s][5] * no3 + x];
        for (int l = 0; l < no; ++l)
          for (int k = 0; k < no; ++k) {
            double acc = 0.0;
            for (int i = 0; i < no; ++i)
              for (int j = 0; j < no; ++j)
                acc += ltv[((size_t)i * no + j) * no + k] * tv[s * no3 + ((size_t)i * no + j) * no + l];
            moo[(size_t)l * no + k] -= 0.5 * acc;
          }
      }
    }
#pragma omp critical
    {
      for (size_t x = 0; x < (size_t)no * no; ++x) doo[x] += moo[x];
    }
    free(Bt); free(Bx); free(tv); free(lv); free(ltv); free(moo);
  }
  memcpy(Doo, doo, (size_t)no * no * sizeof(double));
  memcpy(Dov, dov, n1 * sizeof(double));
  memcpy(Dvv, dvv, nv2 * sizeof(double));
  if (flops) *flops = fl;
  free(V3); free(T); free(lt2); free(Y); free(dvv); free(dov); free(doo);
  return used;
}

/* Only the dressed blocks (for tests that pin them on their own). */
void oracle_dressed_blocks(int no, int nv, const double *chol_L, int naux,
                           const double *R1, double *hvvvo, double *hoovo,
                           double *hooov, double *hvvov, double *hF) {
  dressed_blocks(no, nv, chol_L, naux, R1, hvvvo, hoovo, hooov, hvvov, hF);
}
