/*
 * sx_oracle.c -- plain, slow, CPU FP64 reference ("the oracle") for the
 * atomistic spin effective field, energy and normalised Heun LLG step of
 * arXiv 2605.26016 (SpinX).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library: the
 * neighbour pairs are found here by brute force over lattice translations,
 * the field is the plain pair-list sum, and the thermal noise comes from this
 * file's own Philox4x32-10 and Box-Muller transform.
 *
 * What it follows (Methods section of the paper):
 *   - spin moment mu_i mu_B S_i with |S_i| = 1, energies in meV;
 *   - H_bil = -1/2 sum_{i,j} S_i^T J_ij S_j over directed bonds with
 *     J_ji = J_ij^T (ordered-pair form of the bilinear Hamiltonian);
 *   - J_ij = J I + [[0,Dz,-Dy],[-Dz,0,Dx],[Dy,-Dx,0]] (exchange + DMI tensor);
 *   - H_Z = -sum mu_i mu_B B.S_i ;  H_ani = -sum K (S_i.n)^2 ;
 *   - reduced field b_i = -dH/dS_i in meV, physical field B_i = b_i/(mu_i mu_B);
 *   - pair-list form b_i = sum_{p: i_p = i} J_p S_{j_p} (pair-list backend eq.);
 *   - LLG dS/dt = -gamma/(1+alpha^2) [S x B + alpha S x (S x B)];
 *   - normalised Heun predictor/corrector, N[x] = x/|x|;
 *   - thermal field sigma*eta, sigma = sqrt(2 alpha kB T/(gamma mu mu_B dt)),
 *     the same eta in predictor and corrector (Stratonovich reading);
 *   - dipolar field of point dipoles, O(N^2) direct sum (periodic: minimum
 *     image, a separation of exactly half a period split into its two images
 *     with weight 1/2 each).
 *
 * Units: meV, tesla, fs, nm, kelvin.  Constants (CODATA 2018):
 *   mu_B = 5.7883818060e-2 meV/T, gamma = 1.76085963023e-4 rad/(fs T),
 *   k_B = 8.617333262e-2 meV/K.
 *
 * Site index i = ((s*nz + z)*ny + y)*nx + x; a spin field is stored as three
 * component planes, S[c*nsite + i].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define ORC_MAXSUB 16
#define ORC_MAXSHELL 16
#define ORC_MAXBOND 4096
#define ORC_SEARCH 4 /* cell offsets -4..4 are searched for neighbours */

static const double ORC_MU_B = 5.7883818060e-2;    /* meV / T */
static const double ORC_GAMMA = 1.76085963023e-4;  /* rad / (fs T) */
static const double ORC_K_B = 8.617333262e-2;      /* meV / K */
/* mu0 mu_B^2 / (4 pi) in meV nm^3: 1e-7 T m/A * (9.2740100783e-24 J/T)^2,
 * converted J m^3 -> meV nm^3 by 1e27 / 1.602176634e-22. */
#define ORC_DIP_PREF (1e-7 * 9.2740100783e-24 * 9.2740100783e-24 * 1e27 / 1.602176634e-22)

typedef struct {
  int a, b, d[3];
  double J[9];
} orc_bond;

typedef struct {
  int n[3], pbc[3];
  double A[3][3];
  int nsub;
  double pos[ORC_MAXSUB][3];
  double mu[ORC_MAXSUB];
  int64_t nsite;
  int nshell_req;
  double shellJ[ORC_MAXSHELL];
  int dmi_kind[ORC_MAXSHELL];
  double dmiD[ORC_MAXSHELL];
  int nbond;
  orc_bond bond[ORC_MAXBOND];
  double Bext[3];
  double K[ORC_MAXSUB], nK[ORC_MAXSUB][3];
  int dipolar;
  int nshell;
  double shell_r[256];
  double tol;
  /* pair list, CSR by target site */
  int built;
  int64_t npair;
  int64_t *row, *col;
  double *Jp;
} orc_model;

/* ------------------------------------------------------------------ geometry */

static void cart(const orc_model *m, const double f[3], double out[3]) {
  for (int k = 0; k < 3; k++)
    out[k] = f[0] * m->A[0][k] + f[1] * m->A[1][k] + f[2] * m->A[2][k];
}

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* smallest perpendicular height of the cell: any translation with a cell
 * offset beyond +-M is at least (M-1)*h_min away from every site of a cell */
static double min_height(const orc_model *m) {
  double vol, c[3], best = 1e300;
  const double *a0 = m->A[0], *a1 = m->A[1], *a2 = m->A[2];
  c[0] = a1[1] * a2[2] - a1[2] * a2[1];
  c[1] = a1[2] * a2[0] - a1[0] * a2[2];
  c[2] = a1[0] * a2[1] - a1[1] * a2[0];
  vol = fabs(a0[0] * c[0] + a0[1] * c[1] + a0[2] * c[2]);
  for (int i = 0; i < 3; i++) {
    const double *u = m->A[(i + 1) % 3], *v = m->A[(i + 2) % 3];
    double x[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double h = vol / norm3(x);
    if (h < best) best = h;
  }
  return best;
}

static int cmp_double(const void *x, const void *y) {
  double a = *(const double *)x, b = *(const double *)y;
  return (a > b) - (a < b);
}

/* Distance shells: every distinct distance from a site to another site of the
 * infinite lattice, sorted ascending (ties within m->tol are one shell). */
static void find_shells(orc_model *m) {
  int S = ORC_SEARCH, w = 2 * S + 1;
  int64_t cap = (int64_t)m->nsub * m->nsub * w * w * w;
  double *d = (double *)malloc(sizeof(double) * cap);
  int64_t nd = 0;
  for (int a = 0; a < m->nsub; a++)
    for (int b = 0; b < m->nsub; b++)
      for (int dz = -S; dz <= S; dz++)
        for (int dy = -S; dy <= S; dy++)
          for (int dx = -S; dx <= S; dx++) {
            double f[3] = {dx + m->pos[b][0] - m->pos[a][0], dy + m->pos[b][1] - m->pos[a][1],
                           dz + m->pos[b][2] - m->pos[a][2]};
            double r[3];
            cart(m, f, r);
            double dist = norm3(r);
            if (dist > m->tol) d[nd++] = dist;
          }
  qsort(d, nd, sizeof(double), cmp_double);
  m->nshell = 0;
  for (int64_t i = 0; i < nd && m->nshell < 256; i++)
    if (m->nshell == 0 || d[i] - m->shell_r[m->nshell - 1] > m->tol) m->shell_r[m->nshell++] = d[i];
  free(d);
}

static int shell_of(const orc_model *m, double dist) {
  for (int k = 0; k < m->nshell; k++)
    if (fabs(dist - m->shell_r[k]) <= m->tol) return k;
  return -1;
}

/* ------------------------------------------------------------------ model API */

void *orc_create(const int *n, const int *pbc, const double *A, int nsub, const double *pos,
                 const double *mu) {
  if (nsub < 1 || nsub > ORC_MAXSUB) return NULL;
  for (int k = 0; k < 3; k++)
    if (n[k] < 1) return NULL;
  orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
  double scale = 0;
  for (int k = 0; k < 3; k++) {
    m->n[k] = n[k];
    m->pbc[k] = pbc[k] ? 1 : 0;
    for (int j = 0; j < 3; j++) m->A[k][j] = A[3 * k + j];
    double r = norm3(m->A[k]);
    if (r > scale) scale = r;
  }
  m->nsub = nsub;
  for (int s = 0; s < nsub; s++) {
    for (int j = 0; j < 3; j++) m->pos[s][j] = pos[3 * s + j];
    m->mu[s] = mu[s];
  }
  m->nsite = (int64_t)nsub * n[0] * n[1] * n[2];
  m->tol = 1e-9 * scale;
  find_shells(m);
  return m;
}

static void drop_pairs(orc_model *m) {
  free(m->row);
  free(m->col);
  free(m->Jp);
  m->row = m->col = NULL;
  m->Jp = NULL;
  m->built = 0;
}

void orc_destroy(void *h) {
  orc_model *m = (orc_model *)h;
  if (!m) return;
  drop_pairs(m);
  free(m);
}

int orc_nshell(void *h) { return ((orc_model *)h)->nshell; }
double orc_shell_radius(void *h, int k) {
  orc_model *m = (orc_model *)h;
  return (k >= 0 && k < m->nshell) ? m->shell_r[k] : -1.0;
}

/* shell is 1-based (1 = nearest neighbours) */
int orc_add_shell_exchange(void *h, int shell, double J) {
  orc_model *m = (orc_model *)h;
  if (shell < 1 || shell > ORC_MAXSHELL) return -1;
  if (m->shell_r[shell - 1] > (ORC_SEARCH - 1) * min_height(m)) return -2;
  m->shellJ[shell - 1] += J;
  if (shell > m->nshell_req) m->nshell_req = shell;
  drop_pairs(m);
  return 0;
}

/* kind 0: interfacial, D_ij = D (z x r_ij) on bonds with no z component;
 * kind 1: bulk, D_ij = D r_ij (r_ij unit vector from i to j). */
int orc_add_dmi(void *h, int shell, int kind, double D) {
  orc_model *m = (orc_model *)h;
  if (shell < 1 || shell > ORC_MAXSHELL || (kind != 0 && kind != 1)) return -1;
  if (m->dmiD[shell - 1] != 0.0 && m->dmi_kind[shell - 1] != kind) return -1;
  m->dmi_kind[shell - 1] = kind;
  m->dmiD[shell - 1] += D;
  if (shell > m->nshell_req) m->nshell_req = shell;
  drop_pairs(m);
  return 0;
}

/* Unordered bond: pair energy -S_a(R)^T J S_b(R+d) for every cell R. */
int orc_add_bond(void *h, int a, int b, const int *d, const double *J) {
  orc_model *m = (orc_model *)h;
  if (m->nbond >= ORC_MAXBOND || a < 0 || b < 0 || a >= m->nsub || b >= m->nsub) return -1;
  if (a == b && d[0] == 0 && d[1] == 0 && d[2] == 0) return -1;
  for (int k = 0; k < 3; k++)
    if (abs(d[k]) > ORC_SEARCH) return -2;
  orc_bond *o = &m->bond[m->nbond++];
  o->a = a;
  o->b = b;
  for (int k = 0; k < 3; k++) o->d[k] = d[k];
  for (int k = 0; k < 9; k++) o->J[k] = J[k];
  drop_pairs(m);
  return 0;
}

void orc_set_zeeman(void *h, const double *B) {
  orc_model *m = (orc_model *)h;
  for (int k = 0; k < 3; k++) m->Bext[k] = B[k];
}

int orc_set_anisotropy(void *h, int sub, double K, const double *n) {
  orc_model *m = (orc_model *)h;
  if (sub < 0 || sub >= m->nsub) return -1;
  double r = norm3(n);
  if (!(r > 0)) return -1;
  m->K[sub] = K;
  for (int k = 0; k < 3; k++) m->nK[sub][k] = n[k] / r;
  return 0;
}

void orc_set_dipolar(void *h, int on) { ((orc_model *)h)->dipolar = on ? 1 : 0; }

/* ------------------------------------------------------------------ pair list */

static void site_coords(const orc_model *m, int64_t i, int *s, int c[3]) {
  int64_t t = i;
  c[0] = (int)(t % m->n[0]);
  t /= m->n[0];
  c[1] = (int)(t % m->n[1]);
  t /= m->n[1];
  c[2] = (int)(t % m->n[2]);
  t /= m->n[2];
  *s = (int)t;
}

static int64_t site_index(const orc_model *m, int s, const int c[3]) {
  return (((int64_t)s * m->n[2] + c[2]) * m->n[1] + c[1]) * m->n[0] + c[0];
}

/* All directed bonds into site i, by brute force over every translation within
 * the search box.  Writes up to cap entries; returns the count. */
static int64_t site_pairs(const orc_model *m, int64_t i, int64_t *jout, double *Jout, int64_t cap) {
  int a, c[3];
  site_coords(m, i, &a, c);
  double rmax = (m->nshell_req > 0) ? m->shell_r[m->nshell_req - 1] + m->tol : 0.0;
  int64_t cnt = 0;
  int S = ORC_SEARCH;
  for (int b = 0; b < m->nsub; b++)
    for (int dz = -S; dz <= S; dz++)
      for (int dy = -S; dy <= S; dy++)
        for (int dx = -S; dx <= S; dx++) {
          int dd[3] = {dx, dy, dz};
          double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          int any = 0;
          double f[3] = {dx + m->pos[b][0] - m->pos[a][0], dy + m->pos[b][1] - m->pos[a][1],
                         dz + m->pos[b][2] - m->pos[a][2]};
          double r[3];
          cart(m, f, r);
          double dist = norm3(r);
          if (dist > m->tol && dist <= rmax) {
            int k = shell_of(m, dist);
            if (k >= 0 && k < ORC_MAXSHELL) {
              if (m->shellJ[k] != 0.0) {
                J[0] += m->shellJ[k];
                J[4] += m->shellJ[k];
                J[8] += m->shellJ[k];
                any = 1;
              }
              if (m->dmiD[k] != 0.0) {
                double e[3] = {r[0] / dist, r[1] / dist, r[2] / dist}, D[3];
                int use = 1;
                if (m->dmi_kind[k] == 0) {
                  /* z x e = (-e_y, e_x, 0); only bonds lying in the xy plane */
                  if (fabs(r[2]) > m->tol) use = 0;
                  D[0] = -e[1] * m->dmiD[k];
                  D[1] = e[0] * m->dmiD[k];
                  D[2] = 0.0;
                } else {
                  D[0] = e[0] * m->dmiD[k];
                  D[1] = e[1] * m->dmiD[k];
                  D[2] = e[2] * m->dmiD[k];
                }
                if (use) {
                  /* row alpha of J acting on S_j gives J S_j + S_j x D */
                  J[1] += D[2];
                  J[2] -= D[1];
                  J[3] -= D[2];
                  J[5] += D[0];
                  J[6] += D[1];
                  J[7] -= D[0];
                  any = 1;
                }
              }
            }
          }
          for (int q = 0; q < m->nbond; q++) {
            const orc_bond *o = &m->bond[q];
            if (o->a == a && o->b == b && o->d[0] == dx && o->d[1] == dy && o->d[2] == dz) {
              for (int k = 0; k < 9; k++) J[k] += o->J[k];
              any = 1;
            }
            if (o->b == a && o->a == b && o->d[0] == -dx && o->d[1] == -dy && o->d[2] == -dz) {
              /* reverse directed bond carries the transpose */
              for (int r0 = 0; r0 < 3; r0++)
                for (int c0 = 0; c0 < 3; c0++) J[3 * r0 + c0] += o->J[3 * c0 + r0];
              any = 1;
            }
          }
          if (!any) continue;
          int t[3], ok = 1;
          for (int k = 0; k < 3; k++) {
            t[k] = c[k] + dd[k];
            if (t[k] < 0 || t[k] >= m->n[k]) {
              if (!m->pbc[k]) {
                ok = 0;
                break;
              }
              t[k] = ((t[k] % m->n[k]) + m->n[k]) % m->n[k];
            }
          }
          if (!ok) continue;
          if (cnt < cap) {
            jout[cnt] = site_index(m, b, t);
            for (int k = 0; k < 9; k++) Jout[9 * cnt + k] = J[k];
          }
          cnt++;
        }
  return cnt;
}

#define ORC_PAIRCAP 4096

int orc_build(void *h) {
  orc_model *m = (orc_model *)h;
  drop_pairs(m);
  int64_t N = m->nsite;
  m->row = (int64_t *)malloc(sizeof(int64_t) * (N + 1));
  if (!m->row) return -3;
  int err = 0;
#pragma omp parallel
  {
    int64_t *jj = (int64_t *)malloc(sizeof(int64_t) * ORC_PAIRCAP);
    double *JJ = (double *)malloc(sizeof(double) * 9 * ORC_PAIRCAP);
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < N; i++) {
      int64_t c = site_pairs(m, i, jj, JJ, ORC_PAIRCAP);
      if (c > ORC_PAIRCAP) err = 1;
      m->row[i + 1] = c;
    }
    free(jj);
    free(JJ);
  }
  if (err) return -2;
  m->row[0] = 0;
  for (int64_t i = 0; i < N; i++) m->row[i + 1] += m->row[i];
  m->npair = m->row[N];
  m->col = (int64_t *)malloc(sizeof(int64_t) * (m->npair ? m->npair : 1));
  m->Jp = (double *)malloc(sizeof(double) * 9 * (m->npair ? m->npair : 1));
  if (!m->col || !m->Jp) return -3;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < N; i++)
    site_pairs(m, i, m->col + m->row[i], m->Jp + 9 * m->row[i], m->row[i + 1] - m->row[i]);
  m->built = 1;
  return 0;
}

int64_t orc_npair(void *h) { return ((orc_model *)h)->npair; }

/* Number of directed bonds into site i and their source sites (for tests). */
int64_t orc_site_pairs(void *h, int64_t i, int64_t *jout, double *Jout, int64_t cap) {
  return site_pairs((orc_model *)h, i, jout, Jout, cap);
}

/* ------------------------------------------------------------------ fields */

static void onsite_field(const orc_model *m, int s, const double Si[3], double b[3]) {
  double z = m->mu[s] * ORC_MU_B;
  for (int k = 0; k < 3; k++) b[k] += z * m->Bext[k];
  if (m->K[s] != 0.0) {
    const double *n = m->nK[s];
    double p = Si[0] * n[0] + Si[1] * n[1] + Si[2] * n[2];
    for (int k = 0; k < 3; k++) b[k] += 2.0 * m->K[s] * p * n[k];
  }
}

static void site_pos(const orc_model *m, int64_t i, double r[3]) {
  int s, c[3];
  site_coords(m, i, &s, c);
  double f[3] = {c[0] + m->pos[s][0], c[1] + m->pos[s][1], c[2] + m->pos[s][2]};
  cart(m, f, r);
}

/* Dipolar reduced field at site i, O(N) per site.  Periodic axes use the
 * minimum image in fractional cell coordinates; a separation of exactly half
 * a period is split into its two images with weight 1/2 each. */
static void dipolar_field(const orc_model *m, const double *S, int64_t i, double b[3]) {
  int64_t N = m->nsite;
  int si, ci[3];
  site_coords(m, i, &si, ci);
  for (int64_t j = 0; j < N; j++) {
    if (j == i) continue;
    int sj, cj[3];
    site_coords(m, j, &sj, cj);
    double base[3], w[3][2], off[3][2];
    int nim[3];
    for (int k = 0; k < 3; k++) {
      base[k] = (cj[k] + m->pos[sj][k]) - (ci[k] + m->pos[si][k]);
      nim[k] = 1;
      w[k][0] = 1.0;
      off[k][0] = 0.0;
      if (m->pbc[k]) {
        double L = m->n[k];
        double t = base[k] - L * floor(base[k] / L + 0.5); /* in [-L/2, L/2) */
        if (fabs(fabs(t) - 0.5 * L) < 1e-12) {
          nim[k] = 2;
          w[k][0] = w[k][1] = 0.5;
          off[k][0] = -0.5 * L - base[k];
          off[k][1] = 0.5 * L - base[k];
        } else {
          off[k][0] = t - base[k];
        }
      }
    }
    double pref = ORC_DIP_PREF * m->mu[si] * m->mu[sj];
    for (int ix = 0; ix < nim[0]; ix++)
      for (int iy = 0; iy < nim[1]; iy++)
        for (int iz = 0; iz < nim[2]; iz++) {
          double f[3] = {base[0] + off[0][ix], base[1] + off[1][iy], base[2] + off[2][iz]};
          double r[3];
          cart(m, f, r);
          double d = norm3(r);
          if (d <= m->tol) continue;
          double e[3] = {r[0] / d, r[1] / d, r[2] / d};
          double Sj[3] = {S[j], S[N + j], S[2 * N + j]};
          double es = e[0] * Sj[0] + e[1] * Sj[1] + e[2] * Sj[2];
          double c = pref * w[0][ix] * w[1][iy] * w[2][iz] / (d * d * d);
          for (int k = 0; k < 3; k++) b[k] += c * (3.0 * e[k] * es - Sj[k]);
        }
  }
}

/* bilinear (pair-list) part of the reduced field at site i */
static void bil_field(const orc_model *m, const double *S, int64_t i, double b[3]) {
  int64_t N = m->nsite;
  b[0] = b[1] = b[2] = 0.0;
  for (int64_t p = m->row[i]; p < m->row[i + 1]; p++) {
    int64_t j = m->col[p];
    const double *J = m->Jp + 9 * p;
    double Sj[3] = {S[j], S[N + j], S[2 * N + j]};
    for (int r = 0; r < 3; r++) b[r] += J[3 * r + 0] * Sj[0] + J[3 * r + 1] * Sj[1] + J[3 * r + 2] * Sj[2];
  }
}

static void total_field_site(const orc_model *m, const double *S, int64_t i, double b[3]) {
  int64_t N = m->nsite;
  int s, c[3];
  site_coords(m, i, &s, c);
  bil_field(m, S, i, b);
  double Si[3] = {S[i], S[N + i], S[2 * N + i]};
  onsite_field(m, s, Si, b);
  if (m->dipolar) dipolar_field(m, S, i, b);
}

/* reduced field b (meV) at every site; b has the layout of S */
int orc_field(void *h, const double *S, double *b) {
  orc_model *m = (orc_model *)h;
  if (!m->built) {
    int e = orc_build(m);
    if (e) return e;
  }
  int64_t N = m->nsite;
#pragma omp parallel for schedule(static) if (N > 2048)
  for (int64_t i = 0; i < N; i++) {
    double v[3];
    total_field_site(m, S, i, v);
    b[i] = v[0];
    b[N + i] = v[1];
    b[2 * N + i] = v[2];
  }
  return 0;
}

/* reduced field at selected sites only (no pair list kept): out[3*k + c] */
int orc_field_sites(void *h, const double *S, const int64_t *sites, int64_t nsel, double *out) {
  orc_model *m = (orc_model *)h;
  int64_t N = m->nsite;
  int err = 0;
#pragma omp parallel
  {
    int64_t *jj = (int64_t *)malloc(sizeof(int64_t) * ORC_PAIRCAP);
    double *JJ = (double *)malloc(sizeof(double) * 9 * ORC_PAIRCAP);
#pragma omp for schedule(dynamic, 16)
    for (int64_t k = 0; k < nsel; k++) {
      int64_t i = sites[k];
      if (i < 0 || i >= N) {
        err = 1;
        continue;
      }
      int64_t c = site_pairs(m, i, jj, JJ, ORC_PAIRCAP);
      if (c > ORC_PAIRCAP) {
        err = 1;
        continue;
      }
      double b[3] = {0, 0, 0};
      for (int64_t p = 0; p < c; p++) {
        int64_t j = jj[p];
        const double *J = JJ + 9 * p;
        double Sj[3] = {S[j], S[N + j], S[2 * N + j]};
        for (int r = 0; r < 3; r++) b[r] += J[3 * r] * Sj[0] + J[3 * r + 1] * Sj[1] + J[3 * r + 2] * Sj[2];
      }
      int s, cc[3];
      site_coords(m, i, &s, cc);
      double Si[3] = {S[i], S[N + i], S[2 * N + i]};
      onsite_field(m, s, Si, b);
      if (m->dipolar) dipolar_field(m, S, i, b);
      for (int r = 0; r < 3; r++) out[3 * k + r] = b[r];
    }
    free(jj);
    free(JJ);
  }
  return err ? -1 : 0;
}

/* total energy (meV): E = sum_i [ -1/2 S_i.b_i^bil - mu mu_B B.S_i - K (S_i.n)^2
 *                               - 1/2 S_i.b_i^dip ] ; terms[0..3] receive the parts */
double orc_energy(void *h, const double *S, double *terms) {
  orc_model *m = (orc_model *)h;
  if (!m->built && orc_build(m)) return NAN;
  int64_t N = m->nsite;
  double eb = 0, ez = 0, ea = 0, ed = 0;
#pragma omp parallel for reduction(+ : eb, ez, ea, ed) schedule(static) if (N > 2048)
  for (int64_t i = 0; i < N; i++) {
    int s, c[3];
    site_coords(m, i, &s, c);
    double Si[3] = {S[i], S[N + i], S[2 * N + i]}, b[3];
    bil_field(m, S, i, b);
    eb += -0.5 * (Si[0] * b[0] + Si[1] * b[1] + Si[2] * b[2]);
    ez += -m->mu[s] * ORC_MU_B * (m->Bext[0] * Si[0] + m->Bext[1] * Si[1] + m->Bext[2] * Si[2]);
    if (m->K[s] != 0.0) {
      double p = Si[0] * m->nK[s][0] + Si[1] * m->nK[s][1] + Si[2] * m->nK[s][2];
      ea += -m->K[s] * p * p;
    }
    if (m->dipolar) {
      double d[3] = {0, 0, 0};
      dipolar_field(m, S, i, d);
      ed += -0.5 * (Si[0] * d[0] + Si[1] * d[1] + Si[2] * d[2]);
    }
  }
  if (terms) {
    terms[0] = eb;
    terms[1] = ez;
    terms[2] = ea;
    terms[3] = ed;
  }
  return eb + ez + ea + ed;
}

/* max_i |S_i x b_i| (meV), the torque used as a convergence measure */
double orc_torque_max(void *h, const double *S) {
  orc_model *m = (orc_model *)h;
  int64_t N = m->nsite;
  double *b = (double *)malloc(sizeof(double) * 3 * N);
  if (!b || orc_field(m, S, b)) {
    free(b);
    return NAN;
  }
  double best = 0;
  for (int64_t i = 0; i < N; i++) {
    double s0 = S[i], s1 = S[N + i], s2 = S[2 * N + i];
    double b0 = b[i], b1 = b[N + i], b2 = b[2 * N + i];
    double t0 = s1 * b2 - s2 * b1, t1 = s2 * b0 - s0 * b2, t2 = s0 * b1 - s1 * b0;
    double t = sqrt(t0 * t0 + t1 * t1 + t2 * t2);
    if (t > best) best = t;
  }
  free(b);
  return best;
}

/* ------------------------------------------------------------------ noise */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications with the published multipliers and the key
 * bumped by the published Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* 32 random bits -> uniform in (0,1): (2*(x>>9) + 1) * 2^-24, exact in FP32 */
static float u01(uint32_t x) { return (float)(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f; }

/* natural log of u in (0,1) by u = m 2^e, m in [sqrt(1/2), sqrt(2)],
 * ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9), s = (m-1)/(m+1).
 * Every step is one correctly rounded FP32 operation (built without FP
 * contraction; each Horner step is one fused multiply-add, fmaf, which IEEE 754
 * also rounds once), so the result is reproducible bit for bit. */
static float bm_log(float u) {
  uint32_t bits;
  memcpy(&bits, &u, 4);
  int e = (int)(bits >> 23) - 127;
  uint32_t mb = (bits & 0x007FFFFFu) | 0x3F800000u;
  float mm;
  memcpy(&mm, &mb, 4);
  if (mm > 1.41421356f) {
    mm = mm * 0.5f;
    e = e + 1;
  }
  float s = (mm - 1.0f) / (mm + 1.0f);
  float s2 = s * s;
  float p = 0.111111111f;            /* 1/9 */
  p = fmaf(p, s2, 0.142857143f);     /* 1/7 */
  p = fmaf(p, s2, 0.2f);             /* 1/5 */
  p = fmaf(p, s2, 0.333333333f);     /* 1/3 */
  p = fmaf(p, s2, 1.0f);
  float lnm = (2.0f * s) * p;
  return fmaf((float)e, 0.693147181f, lnm);
}

/* cos and sin of 2 pi u for u in (0,1): quadrant q = floor(4u) (exact),
 * x = (4u - q) pi/2 in [0, pi/2), Taylor series of sin (to x^15) and cos
 * (to x^14) in Horner form with one fmaf per step, then the quadrant map. */
static void bm_sincos2pi(float u, float *cs, float *sn) {
  float t = 4.0f * u;
  int q = (int)t;
  float r = t - (float)q;
  float x = r * 1.57079633f;
  float x2 = x * x;
  float sp = -7.64716373e-13f;            /* -1/15! */
  sp = fmaf(sp, x2, 1.60590438e-10f);     /* 1/13! */
  sp = fmaf(sp, x2, -2.50521084e-8f);     /* -1/11! */
  sp = fmaf(sp, x2, 2.75573192e-6f);      /* 1/9! */
  sp = fmaf(sp, x2, -1.98412698e-4f);     /* -1/7! */
  sp = fmaf(sp, x2, 8.33333333e-3f);      /* 1/5! */
  sp = fmaf(sp, x2, -1.66666667e-1f);     /* -1/3! */
  sp = fmaf(sp, x2, 1.0f);
  float sx = sp * x;
  float cp = -1.14707456e-11f;            /* -1/14! */
  cp = fmaf(cp, x2, 2.08767570e-9f);      /* 1/12! */
  cp = fmaf(cp, x2, -2.75573192e-7f);     /* -1/10! */
  cp = fmaf(cp, x2, 2.48015873e-5f);      /* 1/8! */
  cp = fmaf(cp, x2, -1.38888889e-3f);     /* -1/6! */
  cp = fmaf(cp, x2, 4.16666667e-2f);      /* 1/4! */
  cp = fmaf(cp, x2, -0.5f);               /* -1/2! */
  cp = fmaf(cp, x2, 1.0f);
  float cx = cp;
  switch (q & 3) {
    case 0: *cs = cx; *sn = sx; break;
    case 1: *cs = -sx; *sn = cx; break;
    case 2: *cs = -cx; *sn = -sx; break;
    default: *cs = sx; *sn = -cx; break;
  }
}

/* Three standard normals for (seed, replica, site, step): Philox counter
 * (site_lo, site_hi, step_lo, replica<<8), key (seed_lo, seed_hi); the four
 * words give u0..u3; eta0, eta1 = Box-Muller(u0, u1), eta2 = r(u2) cos(2 pi u3). */
void orc_normals(uint64_t seed, uint32_t replica, uint64_t site, uint64_t step, float *eta) {
  uint32_t ctr[4] = {(uint32_t)site, (uint32_t)(site >> 32), (uint32_t)step, replica << 8};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  float u0 = u01(x[0]), u1 = u01(x[1]), u2 = u01(x[2]), u3 = u01(x[3]);
  float c, s, c2, s2;
  float r0 = sqrtf(-2.0f * bm_log(u0));
  bm_sincos2pi(u1, &c, &s);
  float r1 = sqrtf(-2.0f * bm_log(u2));
  bm_sincos2pi(u3, &c2, &s2);
  eta[0] = r0 * c;
  eta[1] = r0 * s;
  eta[2] = r1 * c2;
}

/* normals for a block of sites (tests) */
void orc_normals_block(uint64_t seed, uint32_t replica, uint64_t site0, int64_t n, uint64_t step, float *eta) {
  for (int64_t k = 0; k < n; k++) orc_normals(seed, replica, site0 + (uint64_t)k, step, eta + 3 * k);
}

/* ------------------------------------------------------------------ dynamics */

/* LLG right-hand side f = -gamma/(1+alpha^2) [S x B + alpha S x (S x B)] */
static void llg_rhs(const double S[3], const double B[3], double alpha, double f[3]) {
  double g = -ORC_GAMMA / (1.0 + alpha * alpha);
  double t[3] = {S[1] * B[2] - S[2] * B[1], S[2] * B[0] - S[0] * B[2], S[0] * B[1] - S[1] * B[0]};
  double u[3] = {S[1] * t[2] - S[2] * t[1], S[2] * t[0] - S[0] * t[2], S[0] * t[1] - S[1] * t[0]};
  for (int k = 0; k < 3; k++) f[k] = g * (t[k] + alpha * u[k]);
}

static void normalise(double x[3]) {
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  x[0] /= r;
  x[1] /= r;
  x[2] /= r;
}

/* nsteps normalised Heun steps in place on S (steps step0 .. step0+nsteps-1).
 * T > 0 adds the thermal field sigma eta with one eta per site and step,
 * shared by predictor and corrector. */
int orc_heun(void *h, double *S, double dt, double alpha, double T, uint64_t seed, uint32_t replica,
             uint64_t step0, int64_t nsteps) {
  orc_model *m = (orc_model *)h;
  if (!m->built) {
    int e = orc_build(m);
    if (e) return e;
  }
  int64_t N = m->nsite;
  double *b = (double *)malloc(sizeof(double) * 3 * N);
  double *St = (double *)malloc(sizeof(double) * 3 * N);
  double *f0 = (double *)malloc(sizeof(double) * 3 * N);
  double *Bth = (double *)malloc(sizeof(double) * 3 * N);
  if (!b || !St || !f0 || !Bth) {
    free(b);
    free(St);
    free(f0);
    free(Bth);
    return -3;
  }
  for (int64_t n = 0; n < nsteps; n++) {
    uint64_t step = step0 + (uint64_t)n;
#pragma omp parallel for schedule(static) if (N > 2048)
    for (int64_t i = 0; i < N; i++) {
      int s, c[3];
      site_coords(m, i, &s, c);
      double th[3] = {0, 0, 0};
      if (T > 0.0) {
        double sigma = sqrt(2.0 * alpha * ORC_K_B * T / (ORC_GAMMA * m->mu[s] * ORC_MU_B * dt));
        float eta[3];
        orc_normals(seed, replica, (uint64_t)i, step, eta);
        for (int k = 0; k < 3; k++) th[k] = sigma * (double)eta[k];
      }
      for (int k = 0; k < 3; k++) Bth[k * N + i] = th[k];
    }
    orc_field(m, S, b);
#pragma omp parallel for schedule(static) if (N > 2048)
    for (int64_t i = 0; i < N; i++) {
      int s, c[3];
      site_coords(m, i, &s, c);
      double mm = m->mu[s] * ORC_MU_B;
      double Si[3] = {S[i], S[N + i], S[2 * N + i]}, B[3], f[3], x[3];
      for (int k = 0; k < 3; k++) B[k] = b[k * N + i] / mm + Bth[k * N + i];
      llg_rhs(Si, B, alpha, f);
      for (int k = 0; k < 3; k++) {
        f0[k * N + i] = f[k];
        x[k] = Si[k] + dt * f[k];
      }
      normalise(x);
      for (int k = 0; k < 3; k++) St[k * N + i] = x[k];
    }
    orc_field(m, St, b);
#pragma omp parallel for schedule(static) if (N > 2048)
    for (int64_t i = 0; i < N; i++) {
      int s, c[3];
      site_coords(m, i, &s, c);
      double mm = m->mu[s] * ORC_MU_B;
      double Sp[3] = {St[i], St[N + i], St[2 * N + i]}, B[3], f[3], x[3];
      for (int k = 0; k < 3; k++) B[k] = b[k * N + i] / mm + Bth[k * N + i];
      llg_rhs(Sp, B, alpha, f);
      for (int k = 0; k < 3; k++) x[k] = S[k * N + i] + 0.5 * dt * (f0[k * N + i] + f[k]);
      normalise(x);
      for (int k = 0; k < 3; k++) S[k * N + i] = x[k];
    }
  }
  free(b);
  free(St);
  free(f0);
  free(Bth);
  return 0;
}

/* One Heun step evaluated only at the selected sites (same arithmetic as
 * orc_heun): the predictor is formed for each selected site and for every
 * source of its bonds, then the corrector at the site.  For checks on large
 * lattices where a full step on the CPU is too slow.  out[3*k + c]. */
int orc_heun_sites(void *h, const double *S, double dt, double alpha, double T, uint64_t seed, uint32_t replica,
                   uint64_t step, const int64_t *sites, int64_t nsel, double *out) {
  orc_model *m = (orc_model *)h;
  if (m->dipolar) return -1;
  int64_t N = m->nsite;
  int err = 0;
#pragma omp parallel
  {
    int64_t *jj = (int64_t *)malloc(sizeof(int64_t) * ORC_PAIRCAP);
    double *JJ = (double *)malloc(sizeof(double) * 9 * ORC_PAIRCAP);
    int64_t *kk = (int64_t *)malloc(sizeof(int64_t) * ORC_PAIRCAP);
    double *KK = (double *)malloc(sizeof(double) * 9 * ORC_PAIRCAP);
    double *St = (double *)malloc(sizeof(double) * 3 * (ORC_PAIRCAP + 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < nsel; q++) {
      int64_t i = sites[q];
      if (i < 0 || i >= N) {
        err = 1;
        continue;
      }
      int64_t ci = site_pairs(m, i, jj, JJ, ORC_PAIRCAP);
      if (ci > ORC_PAIRCAP) {
        err = 1;
        continue;
      }
      double f0i[3];
      /* predictor for the site itself (slot ci) and every bond source (slots 0..ci-1) */
      for (int64_t p = 0; p <= ci; p++) {
        int64_t j = (p < ci) ? jj[p] : i;
        int64_t cj = site_pairs(m, j, kk, KK, ORC_PAIRCAP);
        double b[3] = {0, 0, 0};
        for (int64_t r = 0; r < cj; r++) {
          int64_t k = kk[r];
          const double *J = KK + 9 * r;
          double Sk[3] = {S[k], S[N + k], S[2 * N + k]};
          for (int a = 0; a < 3; a++) b[a] += J[3 * a] * Sk[0] + J[3 * a + 1] * Sk[1] + J[3 * a + 2] * Sk[2];
        }
        int s, cc[3];
        site_coords(m, j, &s, cc);
        double Sj[3] = {S[j], S[N + j], S[2 * N + j]};
        onsite_field(m, s, Sj, b);
        double mm = m->mu[s] * ORC_MU_B, B[3], f[3], x[3], th[3] = {0, 0, 0};
        if (T > 0.0) {
          double sigma = sqrt(2.0 * alpha * ORC_K_B * T / (ORC_GAMMA * m->mu[s] * ORC_MU_B * dt));
          float eta[3];
          orc_normals(seed, replica, (uint64_t)j, step, eta);
          for (int a = 0; a < 3; a++) th[a] = sigma * (double)eta[a];
        }
        for (int a = 0; a < 3; a++) B[a] = b[a] / mm + th[a];
        llg_rhs(Sj, B, alpha, f);
        for (int a = 0; a < 3; a++) x[a] = Sj[a] + dt * f[a];
        normalise(x);
        for (int a = 0; a < 3; a++) St[3 * p + a] = x[a];
        if (p == ci)
          for (int a = 0; a < 3; a++) f0i[a] = f[a];
      }
      /* corrector at the site from the predicted neighbours */
      double b[3] = {0, 0, 0};
      for (int64_t p = 0; p < ci; p++) {
        const double *J = JJ + 9 * p;
        const double *Sp = St + 3 * p;
        for (int a = 0; a < 3; a++) b[a] += J[3 * a] * Sp[0] + J[3 * a + 1] * Sp[1] + J[3 * a + 2] * Sp[2];
      }
      int s, cc[3];
      site_coords(m, i, &s, cc);
      double Sti[3] = {St[3 * ci], St[3 * ci + 1], St[3 * ci + 2]};
      onsite_field(m, s, Sti, b);
      double mm = m->mu[s] * ORC_MU_B, B[3], f[3], x[3], th[3] = {0, 0, 0};
      if (T > 0.0) {
        double sigma = sqrt(2.0 * alpha * ORC_K_B * T / (ORC_GAMMA * m->mu[s] * ORC_MU_B * dt));
        float eta[3];
        orc_normals(seed, replica, (uint64_t)i, step, eta);
        for (int a = 0; a < 3; a++) th[a] = sigma * (double)eta[a];
      }
      for (int a = 0; a < 3; a++) B[a] = b[a] / mm + th[a];
      llg_rhs(Sti, B, alpha, f);
      for (int a = 0; a < 3; a++) x[a] = S[a * N + i] + 0.5 * dt * (f0i[a] + f[a]);
      normalise(x);
      for (int a = 0; a < 3; a++) out[3 * q + a] = x[a];
    }
    free(jj);
    free(JJ);
    free(kk);
    free(KK);
    free(St);
  }
  return err ? -1 : 0;
}

/* ------------------------------------------------------------------ minimisation */

/* Exponential-map retraction ("Static optimization and minimum-energy paths"):
 * R(S, u) = cos|u| S + sin|u| u/|u| for a tangent u (limit S for |u| = 0). */
static void retract_exp(double S[3], const double u[3]) {
  double a = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (a == 0.0) return;
  double c = cos(a), s = sin(a) / a;
  for (int k = 0; k < 3; k++) S[k] = c * S[k] + s * u[k];
  normalise(S);
}

/* Velocity-projection minimisation, niter iterations, in place on S.
 * Force f = b - (b.S) S (tangent part of -dH/dS).  Each iteration:
 *   v <- v + dt/2 (f_prev + f)            (skipped on the first iteration: v = 0)
 *   v <- max(v.f, 0) / (f.f) * f          (sums over the whole system)
 *   S <- R_exp(S, dt v + dt^2/2 f)
 * vstate (3N) and fprev (3N) carry v and f between calls; *first = 1 starts afresh. */
int orc_vp(void *h, double *S, double dt, int64_t niter, double *vstate, double *fprev, int first) {
  orc_model *m = (orc_model *)h;
  if (!m->built) {
    int e = orc_build(m);
    if (e) return e;
  }
  int64_t N = m->nsite;
  double *b = (double *)malloc(sizeof(double) * 3 * N);
  double *f = (double *)malloc(sizeof(double) * 3 * N);
  if (!b || !f) {
    free(b);
    free(f);
    return -3;
  }
  for (int64_t it = 0; it < niter; it++) {
    orc_field(m, S, b);
    double p = 0.0, F2 = 0.0;
    for (int64_t i = 0; i < N; i++) {
      double Si[3] = {S[i], S[N + i], S[2 * N + i]}, bi[3] = {b[i], b[N + i], b[2 * N + i]};
      double d = bi[0] * Si[0] + bi[1] * Si[1] + bi[2] * Si[2];
      for (int k = 0; k < 3; k++) {
        double fk = bi[k] - d * Si[k];
        f[k * N + i] = fk;
        double vk = (first && it == 0) ? 0.0 : vstate[k * N + i] + 0.5 * dt * (fprev[k * N + i] + fk);
        vstate[k * N + i] = vk;
        p += vk * fk;
        F2 += fk * fk;
      }
    }
    double c = (p > 0.0 && F2 > 0.0) ? p / F2 : 0.0;
    for (int64_t i = 0; i < N; i++) {
      double Si[3] = {S[i], S[N + i], S[2 * N + i]}, u[3];
      for (int k = 0; k < 3; k++) {
        double fk = f[k * N + i];
        vstate[k * N + i] = c * fk;
        fprev[k * N + i] = fk;
        u[k] = dt * c * fk + 0.5 * dt * dt * fk;
      }
      retract_exp(Si, u);
      for (int k = 0; k < 3; k++) S[k * N + i] = Si[k];
    }
  }
  free(b);
  free(f);
  return 0;
}

/* ------------------------------------------------------------------ minimum-energy paths */

/* geodesic distance between two spin fields ("Static optimization and
 * minimum-energy paths"): d = [ sum_i arccos^2(S_i^(n).S_i^(m)) ]^(1/2) */
double orc_geodesic(int64_t N, const double *A, const double *B) {
  double s = 0.0;
  for (int64_t i = 0; i < N; i++) {
    double d = A[i] * B[i] + A[N + i] * B[N + i] + A[2 * N + i] * B[2 * N + i];
    if (d > 1.0) d = 1.0;
    if (d < -1.0) d = -1.0;
    double a = acos(d);
    s += a * a;
  }
  return sqrt(s);
}

/* tangent-space projection at S: x - (x.S) S */
static void project(const double S[3], double x[3]) {
  double d = x[0] * S[0] + x[1] * S[1] + x[2] * S[2];
  for (int k = 0; k < 3; k++) x[k] -= d * S[k];
}

/* niter GNEB iterations on a chain of nimg images (img[n*3N ...]); endpoints fixed.
 * Tangent: energy-weighted upwind combination of the projected differences
 * t+ = P(S_{n+1} - S_n), t- = P(S_n - S_{n-1}), normalised over the image.
 * Force on an interior image: f - (f.tau) tau + k (d_{n,n+1} - d_{n-1,n}) tau,
 * or f - 2 (f.tau) tau for the climbing image (the highest-energy interior image
 * when climbing != 0); f = b - (b.S) S.  Update S <- R_exp(S, dt F).
 * E receives the image energies and *fmax_out the largest site force of the last iteration. */
/* GNEB / CI-GNEB forces of every interior image of a chain: E receives the image
 * energies, F (nimg x 3N, interior slots) the forces, *worst the largest site |F|. */
static void gneb_forces(orc_model *m, const double *img, int nimg, double kspring, int climbing, double *E,
                        double *F, double *b, double *worst_out) {
  int64_t N = m->nsite;
  for (int n = 0; n < nimg; n++) E[n] = orc_energy(m, img + (int64_t)n * 3 * N, NULL);
  int top = 1;
  for (int n = 1; n < nimg - 1; n++)
    if (E[n] > E[top]) top = n;
  double worst = 0.0;
  for (int n = 1; n < nimg - 1; n++) {
    const double *S = img + (int64_t)n * 3 * N, *Sp = S + 3 * N, *Sm = S - 3 * N;
    orc_field(m, S, b);
    double a, bb;
    double dEp = E[n + 1] - E[n], dEm = E[n - 1] - E[n];
    if (E[n + 1] > E[n] && E[n] > E[n - 1]) {
      a = 1.0;
      bb = 0.0;
    } else if (E[n + 1] < E[n] && E[n] < E[n - 1]) {
      a = 0.0;
      bb = 1.0;
    } else {
      double emax = fmax(fabs(dEp), fabs(dEm)), emin = fmin(fabs(dEp), fabs(dEm));
      if (E[n + 1] > E[n - 1]) {
        a = emax;
        bb = emin;
      } else {
        a = emin;
        bb = emax;
      }
    }
    double tt = 0.0, ft = 0.0;
    double *tau = F + (int64_t)n * 3 * N; /* tau stored temporarily in F */
    for (int64_t i = 0; i < N; i++) {
      double s[3] = {S[i], S[N + i], S[2 * N + i]}, tp[3], tm[3], bi[3] = {b[i], b[N + i], b[2 * N + i]};
      for (int k = 0; k < 3; k++) {
        tp[k] = Sp[k * N + i] - s[k];
        tm[k] = s[k] - Sm[k * N + i];
      }
      project(s, tp);
      project(s, tm);
      project(s, bi);
      for (int k = 0; k < 3; k++) {
        double t = a * tp[k] + bb * tm[k];
        tau[k * N + i] = t;
        tt += t * t;
        ft += bi[k] * t;
      }
    }
    double tn = sqrt(tt);
    double ftau = tn > 0 ? ft / tn : 0.0;
    double dpl = orc_geodesic(N, S, Sp), dmi = orc_geodesic(N, Sm, S);
    int ci = climbing && n == top;
    double cf = ci ? 2.0 : 1.0, ks = ci ? 0.0 : kspring * (dpl - dmi);
    for (int64_t i = 0; i < N; i++) {
      double s[3] = {S[i], S[N + i], S[2 * N + i]}, bi[3] = {b[i], b[N + i], b[2 * N + i]}, f2 = 0.0;
      project(s, bi);
      for (int k = 0; k < 3; k++) {
        double th = tn > 0 ? tau[k * N + i] / tn : 0.0;
        double Fk = bi[k] - cf * ftau * th + ks * th;
        tau[k * N + i] = Fk;
        f2 += Fk * Fk;
      }
      if (sqrt(f2) > worst) worst = sqrt(f2);
    }
  }
  *worst_out = worst;
}

/* niter GNEB iterations on a chain of nimg images (img[n*3N ...]); endpoints fixed.
 * Tangent: energy-weighted upwind combination of the projected differences
 * t+ = P(S_{n+1} - S_n), t- = P(S_n - S_{n-1}), normalised over the image.
 * Force on an interior image: f - (f.tau) tau + k (d_{n,n+1} - d_{n-1,n}) tau,
 * or f - 2 (f.tau) tau for the climbing image (the highest-energy interior image
 * when climbing != 0); f = b - (b.S) S.  Update S <- R_exp(S, dt F).
 * E receives the image energies and *fmax_out the largest site force of the last iteration. */
int orc_gneb(void *h, double *img, int nimg, double dt, double kspring, int climbing, int64_t niter, double *E,
             double *fmax_out) {
  orc_model *m = (orc_model *)h;
  if (!m->built) {
    int e = orc_build(m);
    if (e) return e;
  }
  if (nimg < 3) return -1;
  int64_t N = m->nsite;
  double *b = (double *)malloc(sizeof(double) * 3 * N);
  double *F = (double *)malloc(sizeof(double) * 3 * N * nimg);
  if (!b || !F) {
    free(b);
    free(F);
    return -3;
  }
  for (int64_t it = 0; it < niter; it++) {
    double worst;
    gneb_forces(m, img, nimg, kspring, climbing, E, F, b, &worst);
    for (int n = 1; n < nimg - 1; n++) {
      double *S = img + (int64_t)n * 3 * N, *Fn = F + (int64_t)n * 3 * N;
      for (int64_t i = 0; i < N; i++) {
        double s[3] = {S[i], S[N + i], S[2 * N + i]}, u[3];
        for (int k = 0; k < 3; k++) u[k] = dt * Fn[k * N + i];
        retract_exp(s, u);
        for (int k = 0; k < 3; k++) S[k * N + i] = s[k];
      }
    }
    *fmax_out = worst;
  }
  for (int n = 0; n < nimg; n++) E[n] = orc_energy(m, img + (int64_t)n * 3 * N, NULL);
  free(b);
  free(F);
  return 0;
}

/* niter GNEB iterations with velocity projection ("Static optimization and
 * minimum-energy paths": velocity projection, Bitzek et al.) on the GNEB force
 * F of all interior images taken as one vector: v' = v + dt/2 (F_prev + F)
 * (v' = 0 on the first iteration when first != 0), c = max(v'.F, 0) / (F.F)
 * with the dot products over every interior image and site, v <- c F,
 * S <- R_exp(S, dt c F + dt^2/2 F), F_prev <- F.  vstate and fprev hold
 * nimg x 3N doubles (interior slots used) and carry the velocity between calls. */
int orc_gneb_vp(void *h, double *img, int nimg, double dt, double kspring, int climbing, int64_t niter, double *E,
                double *fmax_out, double *vstate, double *fprev, int first) {
  orc_model *m = (orc_model *)h;
  if (!m->built) {
    int e = orc_build(m);
    if (e) return e;
  }
  if (nimg < 3) return -1;
  int64_t N = m->nsite;
  double *b = (double *)malloc(sizeof(double) * 3 * N);
  double *F = (double *)malloc(sizeof(double) * 3 * N * nimg);
  if (!b || !F) {
    free(b);
    free(F);
    return -3;
  }
  for (int64_t it = 0; it < niter; it++) {
    double worst;
    gneb_forces(m, img, nimg, kspring, climbing, E, F, b, &worst);
    double p = 0.0, F2 = 0.0;
    for (int n = 1; n < nimg - 1; n++) {
      double *Fn = F + (int64_t)n * 3 * N, *vn = vstate + (int64_t)n * 3 * N, *pn = fprev + (int64_t)n * 3 * N;
      for (int64_t j = 0; j < 3 * N; j++) {
        double vk = (first && it == 0) ? 0.0 : vn[j] + 0.5 * dt * (pn[j] + Fn[j]);
        p += vk * Fn[j];
        F2 += Fn[j] * Fn[j];
      }
    }
    double c = (p > 0.0 && F2 > 0.0) ? p / F2 : 0.0;
    for (int n = 1; n < nimg - 1; n++) {
      double *S = img + (int64_t)n * 3 * N, *Fn = F + (int64_t)n * 3 * N;
      double *vn = vstate + (int64_t)n * 3 * N, *pn = fprev + (int64_t)n * 3 * N;
      for (int64_t i = 0; i < N; i++) {
        double s[3] = {S[i], S[N + i], S[2 * N + i]}, u[3];
        for (int k = 0; k < 3; k++) {
          double fk = Fn[k * N + i];
          vn[k * N + i] = c * fk;
          pn[k * N + i] = fk;
          u[k] = dt * c * fk + 0.5 * dt * dt * fk;
        }
        retract_exp(s, u);
        for (int k = 0; k < 3; k++) S[k * N + i] = s[k];
      }
    }
    *fmax_out = worst;
  }
  for (int n = 0; n < nimg; n++) E[n] = orc_energy(m, img + (int64_t)n * 3 * N, NULL);
  free(b);
  free(F);
  return 0;
}

/* niter string-method iterations: every interior image steps along its tangent
 * force, S <- R_exp(S, dt f), then the images are redistributed at equal
 * geodesic arc length by per-site spherical interpolation between neighbours.
 * *fmax_out receives the largest site force |f| of the last iteration. */
int orc_string(void *h, double *img, int nimg, double dt, int64_t niter, double *E, double *fmax_out) {
  orc_model *m = (orc_model *)h;
  if (!m->built) {
    int e = orc_build(m);
    if (e) return e;
  }
  if (nimg < 3) return -1;
  int64_t N = m->nsite;
  double *b = (double *)malloc(sizeof(double) * 3 * N);
  double *old = (double *)malloc(sizeof(double) * 3 * N * nimg);
  double *L = (double *)malloc(sizeof(double) * nimg);
  if (!b || !old || !L) {
    free(b);
    free(old);
    free(L);
    return -3;
  }
  for (int64_t it = 0; it < niter; it++) {
    double worst = 0.0;
    for (int n = 1; n < nimg - 1; n++) {
      double *S = img + (int64_t)n * 3 * N;
      orc_field(m, S, b);
      for (int64_t i = 0; i < N; i++) {
        double s[3] = {S[i], S[N + i], S[2 * N + i]}, u[3] = {b[i], b[N + i], b[2 * N + i]};
        project(s, u);
        double f = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (f > worst) worst = f;
        for (int k = 0; k < 3; k++) u[k] *= dt;
        retract_exp(s, u);
        for (int k = 0; k < 3; k++) S[k * N + i] = s[k];
      }
    }
    *fmax_out = worst;
    memcpy(old, img, sizeof(double) * 3 * N * nimg);
    L[0] = 0.0;
    for (int n = 1; n < nimg; n++)
      L[n] = L[n - 1] + orc_geodesic(N, old + (int64_t)(n - 1) * 3 * N, old + (int64_t)n * 3 * N);
    for (int n = 1; n < nimg - 1; n++) {
      double target = L[nimg - 1] * n / (nimg - 1);
      int j = 0;
      while (j < nimg - 2 && L[j + 1] < target) j++;
      double seg = L[j + 1] - L[j];
      double w = seg > 0 ? (target - L[j]) / seg : 0.0;
      const double *A = old + (int64_t)j * 3 * N, *B = old + (int64_t)(j + 1) * 3 * N;
      double *S = img + (int64_t)n * 3 * N;
      for (int64_t i = 0; i < N; i++) {
        double a[3] = {A[i], A[N + i], A[2 * N + i]}, c[3] = {B[i], B[N + i], B[2 * N + i]}, s[3];
        double d = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
        if (d > 1.0) d = 1.0;
        if (d < -1.0) d = -1.0;
        double th = acos(d);
        if (th < 1e-12) {
          for (int k = 0; k < 3; k++) s[k] = a[k];
        } else {
          double p = sin((1.0 - w) * th) / sin(th), q = sin(w * th) / sin(th);
          for (int k = 0; k < 3; k++) s[k] = p * a[k] + q * c[k];
        }
        normalise(s);
        for (int k = 0; k < 3; k++) S[k * N + i] = s[k];
      }
    }
  }
  for (int n = 0; n < nimg; n++) E[n] = orc_energy(m, img + (int64_t)n * 3 * N, NULL);
  free(b);
  free(old);
  free(L);
  return 0;
}

int orc_num_threads(void) { return omp_get_max_threads(); }

/* physical constants as used here, for tests */
void orc_constants(double *out) {
  out[0] = ORC_MU_B;
  out[1] = ORC_GAMMA;
  out[2] = ORC_K_B;
  out[3] = ORC_DIP_PREF;
}
