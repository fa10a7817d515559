/*
 * adgref.c -- plain FP64 CPU oracle for the ADG method of arXiv 2603.28710.
 *
 * TEST INFRASTRUCTURE ONLY (see adgref.h).  Slow on purpose: every element residual is
 * a dense quadrature of the weak form over all n^d x n^d basis/point pairs, the mass
 * matrix is assembled and solved by Gaussian elimination, and the PE-boundary flux
 * buffers are per element and shifted level by level as Algorithm 3 describes.
 *
 * Readings of the paper taken here (each one listed with its reason in the design notes):
 *  - nodes and quadrature: p+1 Gauss-Legendre points per direction, collocated;
 *  - LLF dissipation parameter exactly as Eq. 9 prints it (1/2 max sqrt(|u|^2 + c^2));
 *  - 2R Runge-Kutta (Eq. 10) with w updated in place; stage abscissae from the tableau;
 *  - AT coefficients from the moment constraints Eq. 15 with r = 1 and fractional k_m;
 *  - flux_buffer shift of Algorithm 3 read as a shift toward older levels;
 *  - random-delay mode: one splitmix64 draw per (step, interface), flux stored every step.
 */
#include "adgref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 9   /* up to degree 8 */

/* ------------------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights (nodal basis of Eq. 4, collocated quadrature).        */
/* Newton iteration on the Legendre polynomial P_n from the Chebyshev-like first guess.   */
/* ------------------------------------------------------------------------------------ */
static void legendre_eval(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  *pn = p1;
  /* (x^2 - 1) P_n'(x) = n (x P_n(x) - P_{n-1}(x)) */
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

int adgref_gauss(int n, double* x, double* w) {
  if (n < 1 || n > MAXN) return -1;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double pn, dpn;
    for (int it = 0; it < 100; ++it) {
      legendre_eval(n, z, &pn, &dpn);
      double dz = pn / dpn;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre_eval(n, z, &pn, &dpn);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
  return 0;
}

/* Lagrange basis polynomial l_a on the nodes x (Eq. 4, tensor-product factor). */
double adgref_lagrange(int n, const double* x, int a, double xi) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != a) v *= (xi - x[j]) / (x[a] - x[j]);
  return v;
}

/* Derivative of l_a by the product rule. */
double adgref_lagrange_deriv(int n, const double* x, int a, double xi) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == a) continue;
    double t = 1.0 / (x[a] - x[k]);
    for (int j = 0; j < n; ++j)
      if (j != a && j != k) t *= (xi - x[j]) / (x[a] - x[j]);
    s += t;
  }
  return s;
}

/* ------------------------------------------------------------------------------------ */
/* Dense linear solve: Gaussian elimination with partial pivoting (used for the AT       */
/* moment system of Eq. 15 and for the element mass matrix of Eq. 7).                    */
/* ------------------------------------------------------------------------------------ */
static int lu_factor(int m, double* A, int* piv) {
  for (int c = 0; c < m; ++c) {
    int best = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[r * m + c]) > fabs(A[best * m + c])) best = r;
    piv[c] = best;
    if (A[best * m + c] == 0.0) return -1;
    if (best != c)
      for (int j = 0; j < m; ++j) {
        double t = A[c * m + j];
        A[c * m + j] = A[best * m + j];
        A[best * m + j] = t;
      }
    for (int r = c + 1; r < m; ++r) {
      double f = A[r * m + c] / A[c * m + c];
      A[r * m + c] = f;
      for (int j = c + 1; j < m; ++j) A[r * m + j] -= f * A[c * m + j];
    }
  }
  return 0;
}

static void lu_solve(int m, const double* LU, const int* piv, double* b) {
  for (int c = 0; c < m; ++c) {
    if (piv[c] != c) {
      double t = b[c];
      b[c] = b[piv[c]];
      b[piv[c]] = t;
    }
  }
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < r; ++j) b[r] -= LU[r * m + j] * b[j];
  for (int r = m - 1; r >= 0; --r) {
    for (int j = r + 1; j < m; ++j) b[r] -= LU[r * m + j] * b[j];
    b[r] /= LU[r * m + r];
  }
}

/* ------------------------------------------------------------------------------------ */
/* AT flux coefficients (Eq. 14-15, r = 1): the N_p+1 weights on the stored levels       */
/* l = k_m, k_m+1, ..., k_m+N_p solve  sum_l c^l (-l dt)^z / z! = [z == 0],  z = 0..N_p.  */
/* dt cancels; k_m may be fractional (naive RK coupling, k_m = k + stage offset).        */
/* ------------------------------------------------------------------------------------ */
int adgref_at_coeffs(int np, double km, double* c) {
  /* The moment matrix is a Vandermonde matrix in -(k_m + l); for N_p >= 4 its condition
     number exceeds 1e6, so Gaussian elimination with partial pivoting is carried out in
     long double to keep the weights accurate to FP64 rounding. */
  int m = np + 1;
  if (np < 0 || m > 16) return -1;
  long double A[256], b[16];
  for (int z = 0; z < m; ++z) {
    long double fact = 1.0L;
    for (int q = 2; q <= z; ++q) fact *= q;
    for (int l = 0; l < m; ++l) {
      long double p = 1.0L;
      for (int q = 0; q < z; ++q) p *= -((long double)km + l);
      A[z * m + l] = p / fact;
    }
    b[z] = (z == 0) ? 1.0L : 0.0L;
  }
  for (int col = 0; col < m; ++col) {
    int best = col;
    for (int r = col + 1; r < m; ++r)
      if (fabsl(A[r * m + col]) > fabsl(A[best * m + col])) best = r;
    if (A[best * m + col] == 0.0L) return -1;
    if (best != col) {
      for (int j = 0; j < m; ++j) {
        long double t = A[col * m + j];
        A[col * m + j] = A[best * m + j];
        A[best * m + j] = t;
      }
      long double t = b[col];
      b[col] = b[best];
      b[best] = t;
    }
    for (int r = col + 1; r < m; ++r) {
      long double f = A[r * m + col] / A[col * m + col];
      for (int j = col; j < m; ++j) A[r * m + j] -= f * A[col * m + j];
      b[r] -= f * b[col];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    long double acc = b[r];
    for (int j = r + 1; j < m; ++j) acc -= A[r * m + j] * b[j];
    b[r] = acc / A[r * m + r];
  }
  for (int l = 0; l < m; ++l) c[l] = (double)b[l];
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Runge-Kutta tables.  LSERK(2,2) and LSERK(3,3): Table 2, 2R form of Eq. 10.            */
/* CK4(5): the 2N scheme of Carpenter & Kennedy (1994), solution 3, not printed in the   */
/* paper.  Butcher arrays are derived from the low-storage coefficients.                  */
/* ------------------------------------------------------------------------------------ */
int adgref_rk_tableau(int scheme, double* a, double* b, double* c, double* ba, double* bb) {
  int s;
  double A[8] = {0}, B[8] = {0};
  double BA[64] = {0}, BB[8] = {0};
  if (scheme == ADGREF_RK22 || scheme == ADGREF_RK33) {
    if (scheme == ADGREF_RK22) {
      s = 2;
      A[0] = 1.0;
      B[0] = 0.5; B[1] = 0.5;
    } else {
      s = 3;
      A[0] = 0.755726352; A[1] = 0.386954477;
      B[0] = 0.245170287; B[1] = 0.184896052; B[2] = 0.569933661;
    }
    /* r_{m+1} = w^{(m)} + dt a_m k_m with w^{(m)} = w^n + dt sum_{j<m} b_j k_j */
    for (int i = 1; i < s; ++i) {
      for (int j = 0; j < i - 1; ++j) BA[i * 8 + j] = B[j];
      BA[i * 8 + i - 1] = A[i - 1];
    }
    for (int j = 0; j < s; ++j) BB[j] = B[j];
  } else if (scheme == ADGREF_CK45) {
    s = 5;
    A[0] = 0.0;
    A[1] = -567301805773.0 / 1357537059087.0;
    A[2] = -2404267990393.0 / 2016746695238.0;
    A[3] = -3550918686646.0 / 2091501179385.0;
    A[4] = -1275806237668.0 / 842570457699.0;
    B[0] = 1432997174477.0 / 9575080441755.0;
    B[1] = 5161836677717.0 / 13612068292357.0;
    B[2] = 1720146321549.0 / 2090206949498.0;
    B[3] = 3134564353537.0 / 4481467310338.0;
    B[4] = 2277821191437.0 / 14882151754819.0;
    /* q_i = A_i q_{i-1} + dt k_i ; w_i = w_{i-1} + B_i q_i.
       Stage i+1 sees w_i = w^n + dt sum_{j<=i} k_j sum_{m=j..i} B_m prod_{l=j+1..m} A_l. */
    for (int i = 0; i < s; ++i) {
      for (int j = 0; j <= i; ++j) {
        double acc = 0.0;
        for (int m = j; m <= i; ++m) {
          double prod = 1.0;
          for (int l = j + 1; l <= m; ++l) prod *= A[l];
          acc += B[m] * prod;
        }
        if (i + 1 < s) BA[(i + 1) * 8 + j] = acc;
        else BB[j] = acc;
      }
    }
  } else {
    return -1;
  }
  for (int i = 0; i < s; ++i) {
    double ci = 0.0;
    for (int j = 0; j < i; ++j) ci += BA[i * 8 + j];
    if (a) a[i] = A[i];
    if (b) b[i] = B[i];
    if (c) c[i] = ci;
    if (bb) bb[i] = BB[i];
    if (ba)
      for (int j = 0; j < s; ++j) ba[i * s + j] = BA[i * 8 + j];
  }
  return s;
}

/* ------------------------------------------------------------------------------------ */
/* Euler flux (Eq. 2-3), gravity-free: column `dir` of F(w).                               */
/* ------------------------------------------------------------------------------------ */
void adgref_euler_flux(int dim, double gamma, const double* w, int dir, double* f) {
  double rho = w[0];
  double u[3] = {0.0, 0.0, 0.0}, kin = 0.0;
  for (int d = 0; d < dim; ++d) {
    u[d] = w[1 + d] / rho;
    kin += w[1 + d] * u[d];
  }
  double p = (gamma - 1.0) * (w[dim + 1] - 0.5 * kin);
  f[0] = w[1 + dir];
  for (int d = 0; d < dim; ++d) f[1 + d] = w[1 + d] * u[dir] + (d == dir ? p : 0.0);
  f[dim + 1] = (w[dim + 1] + p) * u[dir];
}

/* Local Lax-Friedrichs flux along the outward normal of the minus side (Eq. 8) with the  */
/* dissipation parameter lambda = 1/2 max(sqrt(|u-|^2 + c-^2), sqrt(|u+|^2 + c+^2)) (Eq. 9). */
void adgref_llf(int dim, double gamma, const double* wm, const double* wp, const double* normal,
                double* fhat) {
  int nv = dim + 2;
  double fm[5], fp[5], fmn[5] = {0}, fpn[5] = {0};
  for (int d = 0; d < dim; ++d) {
    adgref_euler_flux(dim, gamma, wm, d, fm);
    adgref_euler_flux(dim, gamma, wp, d, fp);
    for (int v = 0; v < nv; ++v) {
      fmn[v] += normal[d] * fm[v];
      fpn[v] += normal[d] * fp[v];
    }
  }
  double s2[2];
  const double* ws[2] = {wm, wp};
  for (int side = 0; side < 2; ++side) {
    const double* w = ws[side];
    double rho = w[0], u2 = 0.0, kin = 0.0;
    for (int d = 0; d < dim; ++d) {
      double ud = w[1 + d] / rho;
      u2 += ud * ud;
      kin += w[1 + d] * ud;
    }
    double p = (gamma - 1.0) * (w[dim + 1] - 0.5 * kin);
    double c2 = gamma * p / rho;
    s2[side] = u2 + c2;
  }
  double lambda = 0.5 * fmax(sqrt(s2[0]), sqrt(s2[1]));
  for (int v = 0; v < nv; ++v) fhat[v] = 0.5 * (fmn[v] + fpn[v]) + 0.5 * lambda * (wm[v] - wp[v]);
}

/* ------------------------------------------------------------------------------------ */
/* Schedules: Algorithm 2 (standard flux), Algorithm 3 (AT flux), and the seeded random   */
/* delay mode (one splitmix64 draw per step and subdomain interface).                      */
/* ------------------------------------------------------------------------------------ */
uint64_t adgref_splitmix64(uint64_t x) {
  /* Steele, Lea & Flood (2014): one output of the generator whose state is x. */
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int adgref_num_interfaces(int dim, const int* P) {
  int nsub = 1;
  for (int d = 0; d < dim; ++d) nsub *= P[d];
  int n = 0;
  for (int d = 0; d < dim; ++d)
    if (P[d] > 1) n += nsub;
  return n;
}

static int random_delay(int flux, int np, uint64_t seed, int dmax, int64_t n, int niface,
                        int iface) {
  if (flux == ADGREF_FLUX_SYNC) return 0;
  uint64_t ctr = (uint64_t)n * (uint64_t)niface + (uint64_t)iface;
  int kt = (int)(adgref_splitmix64(seed ^ ctr) % (uint64_t)(dmax + 1));
  int need = (flux == ADGREF_FLUX_STD) ? kt : kt + np;
  if (n - need < 0) kt = 0; /* history not yet long enough: use fresh data */
  return kt;
}

int adgref_schedule(int flux, int delay_mode, int max_delay, int np, const int* P, int dim,
                    uint64_t seed, int dmax, int64_t n0, int count, int32_t* comm, int32_t* k,
                    int32_t* iface_delay) {
  int niface = adgref_num_interfaces(dim, P);
  if (delay_mode == ADGREF_DELAY_RANDOM) {
    for (int i = 0; i < count; ++i) {
      int64_t n = n0 + i;
      int kmax = 0;
      for (int f = 0; f < niface; ++f) {
        int kt = random_delay(flux, np, seed, dmax, n, niface, f);
        if (iface_delay) iface_delay[(int64_t)i * niface + f] = kt;
        if (kt > kmax) kmax = kt;
      }
      comm[i] = (kmax == 0);
      k[i] = kmax;
    }
    return 0;
  }
  /* Literal run of the flag/counter logic from step 0. */
  int kc = 0;
  for (int64_t n = 0; n < n0 + count; ++n) {
    int c;
    if (flux == ADGREF_FLUX_SYNC) c = 1;
    else if (flux == ADGREF_FLUX_STD) c = (n % max_delay) == 0;
    else c = (n % (max_delay + np + 1)) < (np + 1);
    if (c) kc = 0;
    else kc = kc + 1;
    if (n >= n0) {
      comm[n - n0] = c;
      k[n - n0] = kc;
      if (iface_delay)
        for (int f = 0; f < niface; ++f) iface_delay[(n - n0) * niface + f] = kc;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Solver state.                                                                          */
/* ------------------------------------------------------------------------------------ */
struct adgref {
  adgref_params p;
  int dim, nn, nd, nf, nv, nfaces;
  int64_t ne;
  int n[3];
  double h[3];
  double x1[MAXN], w1[MAXN];
  double* phi_vol;  /* [i][q]          phi_i(x_q)                                    */
  double* grad_vol; /* [i][q][d]       d phi_i / d x_d at x_q (physical coordinates)   */
  double* wq;       /* [q]             omega_q |J|                                      */
  double* phi_face; /* [f][i][fq]      phi_i at face point fq of face f                */
  double* wfq;      /* [f][fq]         face weight times face Jacobian                 */
  double* mlu;      /* [i][j]          LU factors of the element mass matrix           */
  int* piv;
  double *w, *r, *kk, *q;
  int64_t step;
  double t;
  int kcount;
  int stages, rk2n;
  double rka[8], rkb[8], rkc[8];
  int np, depth, niface, ntrace;
  int64_t* slot; /* [e][f] -> PE buffer slot or -1 */
  int64_t nslot;
  double* buf;   /* [slot][level][fq][var]: fluxes, or minus-side traces for AT_TRACE */
  double* bufp;  /* plus-side traces for AT_TRACE */
  /* per-stage schedule data */
  int comm;
  int* idelay;   /* [iface] effective delay in random mode */
  double coef[16][16]; /* [delay][l] AT weights for the current stage */
  /* scratch */
  double *F, *V, *S;
};

static int64_t elem_index(const adgref* o, const int* c) {
  int64_t e = 0;
  for (int d = o->dim - 1; d >= 0; --d) e = e * o->n[d] + c[d];
  return e;
}

static void elem_coords(const adgref* o, int64_t e, int* c) {
  for (int d = 0; d < o->dim; ++d) {
    c[d] = (int)(e % o->n[d]);
    e /= o->n[d];
  }
}

static int64_t neighbour(const adgref* o, int64_t e, int dir, int step) {
  int c[3];
  elem_coords(o, e, c);
  c[dir] = (c[dir] + step + o->n[dir]) % o->n[dir];
  return elem_index(o, c);
}

static int subdomain(const adgref* o, int64_t e) {
  int c[3], s = 0;
  elem_coords(o, e, c);
  for (int d = o->dim - 1; d >= 0; --d) s = s * o->p.P[d] + c[d] / (o->n[d] / o->p.P[d]);
  return s;
}

/* reference coordinates of volume point q */
static void vol_point(const adgref* o, int q, double* xi, int* idx) {
  for (int d = 0; d < o->dim; ++d) {
    idx[d] = q % o->nn;
    xi[d] = o->x1[idx[d]];
    q /= o->nn;
  }
}

/* reference coordinates of point fq on face f (dir = f/2, side = f%2: 0 -> xi=-1, 1 -> +1) */
static void face_point(const adgref* o, int f, int fq, double* xi) {
  int dir = f / 2, side = f % 2;
  for (int d = 0; d < o->dim; ++d) {
    if (d == dir) {
      xi[d] = side ? 1.0 : -1.0;
    } else {
      xi[d] = o->x1[fq % o->nn];
      fq /= o->nn;
    }
  }
}

static double basis_at(const adgref* o, int i, const double* xi) {
  double v = 1.0;
  for (int d = 0; d < o->dim; ++d) {
    v *= adgref_lagrange(o->nn, o->x1, i % o->nn, xi[d]);
    i /= o->nn;
  }
  return v;
}

static double basis_grad_at(const adgref* o, int i, const double* xi, int dir) {
  double v = 1.0;
  int ii = i;
  for (int d = 0; d < o->dim; ++d) {
    int a = ii % o->nn;
    ii /= o->nn;
    v *= (d == dir) ? adgref_lagrange_deriv(o->nn, o->x1, a, xi[d])
                    : adgref_lagrange(o->nn, o->x1, a, xi[d]);
  }
  return v * 2.0 / o->h[dir]; /* reference -> physical derivative on the affine element */
}

adgref* adgref_create(const adgref_params* prm) {
  if (prm->dim < 2 || prm->dim > 3 || prm->degree < 1 || prm->degree >= MAXN) return NULL;
  /* Algorithm 2 takes n % L (L >= 1); Algorithm 3 takes n % (L + N_p + 1) (L >= 0). */
  if (prm->delay_mode == ADGREF_DELAY_CAA && prm->max_delay < (prm->flux == ADGREF_FLUX_STD ? 1 : 0))
    return NULL;
  if (prm->delay_mode == ADGREF_DELAY_RANDOM && (prm->random_delay_max < 0 || prm->random_delay_max > 15))
    return NULL;
  adgref* o = (adgref*)calloc(1, sizeof(adgref));
  o->p = *prm;
  o->dim = prm->dim;
  o->nn = prm->degree + 1;
  o->nv = o->dim + 2;
  o->nd = 1;
  o->nf = 1;
  o->ne = 1;
  for (int d = 0; d < o->dim; ++d) {
    o->n[d] = prm->n_elem[d];
    if (o->p.P[d] < 1 || o->n[d] % o->p.P[d] != 0) { free(o); return NULL; }
    o->h[d] = (prm->hi[d] - prm->lo[d]) / o->n[d];
    o->nd *= o->nn;
    o->ne *= o->n[d];
  }
  for (int d = o->dim; d < 3; ++d) { o->n[d] = 1; o->h[d] = 1.0; o->p.P[d] = 1; }
  o->nf = o->nd / o->nn;
  o->nfaces = 2 * o->dim;
  adgref_gauss(o->nn, o->x1, o->w1);
  double J = 1.0;
  for (int d = 0; d < o->dim; ++d) J *= o->h[d] / 2.0;

  int nd = o->nd, nf = o->nf, dim = o->dim;
  o->phi_vol = malloc(sizeof(double) * nd * nd);
  o->grad_vol = malloc(sizeof(double) * nd * nd * 3);
  o->wq = malloc(sizeof(double) * nd);
  o->phi_face = malloc(sizeof(double) * o->nfaces * nd * nf);
  o->wfq = malloc(sizeof(double) * o->nfaces * nf);
  o->mlu = malloc(sizeof(double) * nd * nd);
  o->piv = malloc(sizeof(int) * nd);
  for (int q = 0; q < nd; ++q) {
    double xi[3];
    int idx[3];
    vol_point(o, q, xi, idx);
    double wt = J;
    for (int d = 0; d < dim; ++d) wt *= o->w1[idx[d]];
    o->wq[q] = wt;
    for (int i = 0; i < nd; ++i) {
      o->phi_vol[i * nd + q] = basis_at(o, i, xi);
      for (int d = 0; d < dim; ++d) o->grad_vol[(i * nd + q) * 3 + d] = basis_grad_at(o, i, xi, d);
    }
  }
  for (int f = 0; f < o->nfaces; ++f) {
    int dir = f / 2;
    double Jf = 1.0;
    for (int d = 0; d < dim; ++d)
      if (d != dir) Jf *= o->h[d] / 2.0;
    for (int fq = 0; fq < nf; ++fq) {
      double xi[3];
      face_point(o, f, fq, xi);
      double wt = Jf;
      int t = fq;
      for (int d = 0; d < dim; ++d) {
        if (d == dir) continue;
        wt *= o->w1[t % o->nn];
        t /= o->nn;
      }
      o->wfq[f * nf + fq] = wt;
      for (int i = 0; i < nd; ++i) o->phi_face[(f * nd + i) * nf + fq] = basis_at(o, i, xi);
    }
  }
  /* element mass matrix M_ij = sum_q omega_q |J| phi_i(x_q) phi_j(x_q) (Eq. 7) */
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j < nd; ++j) {
      double s = 0.0;
      for (int q = 0; q < nd; ++q) s += o->wq[q] * o->phi_vol[i * nd + q] * o->phi_vol[j * nd + q];
      o->mlu[i * nd + j] = s;
    }
  lu_factor(nd, o->mlu, o->piv);

  int64_t sz = (int64_t)o->nv * o->ne * nd;
  o->w = calloc(sz, sizeof(double));
  o->r = calloc(sz, sizeof(double));
  o->kk = calloc(sz, sizeof(double));
  o->q = calloc(sz, sizeof(double));

  double ba[64], bb[8];
  o->stages = adgref_rk_tableau(prm->rk, o->rka, o->rkb, o->rkc, ba, bb);
  o->rk2n = (prm->rk == ADGREF_CK45);
  o->np = prm->at_np > 0 ? prm->at_np : prm->degree;
  o->niface = adgref_num_interfaces(dim, o->p.P);
  o->idelay = calloc(o->niface + 1, sizeof(int));

  /* PE-boundary face sides: a face whose two elements lie in different subdomains */
  o->slot = malloc(sizeof(int64_t) * o->ne * o->nfaces);
  o->nslot = 0;
  for (int64_t e = 0; e < o->ne; ++e)
    for (int f = 0; f < o->nfaces; ++f) {
      int64_t nb = neighbour(o, e, f / 2, (f % 2) ? 1 : -1);
      o->slot[e * o->nfaces + f] = (subdomain(o, e) != subdomain(o, nb)) ? o->nslot++ : -1;
    }
  if (prm->flux == ADGREF_FLUX_SYNC) o->depth = 0;
  else if (prm->delay_mode == ADGREF_DELAY_RANDOM)
    o->depth = prm->random_delay_max + (prm->flux == ADGREF_FLUX_STD ? 0 : o->np) + 1;
  else
    o->depth = (prm->flux == ADGREF_FLUX_STD) ? 1 : o->np + 1;
  int64_t bsz = o->nslot * o->depth * nf * o->nv;
  o->buf = calloc(bsz + 1, sizeof(double));
  o->bufp = calloc(prm->flux == ADGREF_FLUX_AT_TRACE ? bsz + 1 : 1, sizeof(double));
  o->F = malloc(sizeof(double) * 3 * o->nv * nd);  /* scratch of the one-element calls */
  o->V = malloc(sizeof(double) * o->nv * nd);
  o->S = malloc(sizeof(double) * o->nv * nd);
  return o;
}

void adgref_destroy(adgref* o) {
  if (!o) return;
  free(o->phi_vol); free(o->grad_vol); free(o->wq); free(o->phi_face); free(o->wfq);
  free(o->mlu); free(o->piv); free(o->w); free(o->r); free(o->kk); free(o->q);
  free(o->idelay); free(o->slot); free(o->buf); free(o->bufp);
  free(o->F); free(o->V); free(o->S);
  free(o);
}

int64_t adgref_state_size(const adgref* o) { return (int64_t)o->nv * o->ne * o->nd; }

void adgref_set_state(adgref* o, const double* u) {
  memcpy(o->w, u, sizeof(double) * adgref_state_size(o));
  o->step = 0;
  o->t = 0.0;
  o->kcount = 0;
}

void adgref_get_state(const adgref* o, double* u) {
  memcpy(u, o->w, sizeof(double) * adgref_state_size(o));
}

/* ------------------------------------------------------------------------------------ */
/* Numerical flux on one face point, with the PE-boundary rules of Algorithms 2 and 3.    */
/* mode: 0 = all fresh (synchronous operator), 1 = schedule of the current step.           */
/* ------------------------------------------------------------------------------------ */
static void extrapolate(const adgref* o, const double* b, int64_t s, int fq, int first,
                        const double* c, double* out) {
  int nf = o->nf, nv = o->nv;
  for (int v = 0; v < nv; ++v) out[v] = 0.0;
  for (int l = 0; l <= o->np; ++l) {
    const double* src = b + ((s * o->depth + first + l) * nf + fq) * nv;
    for (int v = 0; v < nv; ++v) out[v] += c[l] * src[v];
  }
}

static void face_flux(adgref* o, int64_t e, int f, int fq, const double* wm, const double* wp,
                      const double* normal, int stage, int mode, double* fhat) {
  int64_t s = o->slot[e * o->nfaces + f];
  int flux = o->p.flux;
  if (mode == 0 || s < 0 || flux == ADGREF_FLUX_SYNC) {
    adgref_llf(o->dim, o->p.gamma, wm, wp, normal, fhat);
    return;
  }
  int nf = o->nf, nv = o->nv, depth = o->depth;
  int delay;
  int store;
  if (o->p.delay_mode == ADGREF_DELAY_RANDOM) {
    int dir = f / 2;
    int64_t minus = (f % 2) ? e : neighbour(o, e, dir, -1);
    int off = 0;
    int nsub = 1;
    for (int d = 0; d < o->dim; ++d) nsub *= o->p.P[d];
    for (int d = 0; d < dir; ++d)
      if (o->p.P[d] > 1) off += nsub;
    delay = o->idelay[off + subdomain(o, minus)];
    store = (stage == 0); /* every step keeps its stage-0 flux */
  } else {
    delay = o->comm ? 0 : o->kcount;
    store = (stage == 0 && o->comm);
  }
  double fresh[5], tm[5], tp[5];
  adgref_llf(o->dim, o->p.gamma, wm, wp, normal, fresh);
  if (store) {
    /* shift: buffer(l+1) <- buffer(l), oldest level dropped; then buffer(0) <- new */
    for (int l = depth - 1; l >= 1; --l)
      for (int v = 0; v < nv; ++v) {
        o->buf[((s * depth + l) * nf + fq) * nv + v] = o->buf[((s * depth + l - 1) * nf + fq) * nv + v];
        if (flux == ADGREF_FLUX_AT_TRACE)
          o->bufp[((s * depth + l) * nf + fq) * nv + v] =
              o->bufp[((s * depth + l - 1) * nf + fq) * nv + v];
      }
    for (int v = 0; v < nv; ++v) {
      if (flux == ADGREF_FLUX_AT_TRACE) {
        o->buf[((s * depth) * nf + fq) * nv + v] = wm[v];
        o->bufp[((s * depth) * nf + fq) * nv + v] = wp[v];
      } else {
        o->buf[((s * depth) * nf + fq) * nv + v] = fresh[v];
      }
    }
  }
  if (delay == 0) {
    for (int v = 0; v < nv; ++v) fhat[v] = fresh[v];
    return;
  }
  /* In the CAA schedule buffer(0) holds level n-k; in the random mode (stored every step)
     level n-k sits at buffer(k). */
  int first = (o->p.delay_mode == ADGREF_DELAY_RANDOM) ? delay : 0;
  if (flux == ADGREF_FLUX_STD) {
    for (int v = 0; v < nv; ++v) fhat[v] = o->buf[((s * depth + first) * nf + fq) * nv + v];
  } else if (flux == ADGREF_FLUX_AT) {
    extrapolate(o, o->buf, s, fq, first, o->coef[delay], fhat);
  } else {
    extrapolate(o, o->buf, s, fq, first, o->coef[delay], tm);
    extrapolate(o, o->bufp, s, fq, first, o->coef[delay], tp);
    adgref_llf(o->dim, o->p.gamma, tm, tp, normal, fhat);
  }
}

/* ------------------------------------------------------------------------------------ */
/* Element residual k_e = M^{-1} [ (grad phi_i, F(w_h)) - <phi_i, n . F^> ]  (Eq. 6-7),   */
/* by dense quadrature over all basis-function / quadrature-point pairs.                   */
/* ------------------------------------------------------------------------------------ */
/* F, V, S: scratch of 3 nv nd, nv nd and nv nd values (one set per thread). */
static void element_rhs(adgref* o, const double* u, int64_t e, int stage, int mode, double* out,
                        double* F, double* V, double* S) {
  int nd = o->nd, nv = o->nv, dim = o->dim, nf = o->nf;
  int64_t ne = o->ne;
  for (int q = 0; q < nd; ++q) {
    double wv[5], fv[5];
    for (int v = 0; v < nv; ++v) wv[v] = u[(v * ne + e) * nd + q];
    for (int d = 0; d < dim; ++d) {
      adgref_euler_flux(dim, o->p.gamma, wv, d, fv);
      for (int v = 0; v < nv; ++v) F[(d * nv + v) * nd + q] = fv[v];
    }
  }
  for (int v = 0; v < nv; ++v)
    for (int i = 0; i < nd; ++i) {
      double s = 0.0;
      for (int q = 0; q < nd; ++q)
        for (int d = 0; d < dim; ++d)
          s += o->wq[q] * o->grad_vol[(i * nd + q) * 3 + d] * F[(d * nv + v) * nd + q];
      V[v * nd + i] = s;
      S[v * nd + i] = 0.0;
    }
  for (int f = 0; f < o->nfaces; ++f) {
    int dir = f / 2, side = f % 2;
    int64_t nb = neighbour(o, e, dir, side ? 1 : -1);
    int fo = 2 * dir + (1 - side);
    double normal[3] = {0.0, 0.0, 0.0};
    normal[dir] = side ? 1.0 : -1.0;
    for (int fq = 0; fq < nf; ++fq) {
      double wm[5], wp[5], fh[5];
      for (int v = 0; v < nv; ++v) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < nd; ++j) {
          a += u[(v * ne + e) * nd + j] * o->phi_face[(f * nd + j) * nf + fq];
          b += u[(v * ne + nb) * nd + j] * o->phi_face[(fo * nd + j) * nf + fq];
        }
        wm[v] = a;
        wp[v] = b;
      }
      face_flux(o, e, f, fq, wm, wp, normal, stage, mode, fh);
      for (int v = 0; v < nv; ++v)
        for (int i = 0; i < nd; ++i)
          S[v * nd + i] += o->wfq[f * nf + fq] * o->phi_face[(f * nd + i) * nf + fq] * fh[v];
    }
  }
  for (int v = 0; v < nv; ++v) {
    double b[MAXN * MAXN * MAXN];
    for (int i = 0; i < nd; ++i) b[i] = V[v * nd + i] - S[v * nd + i];
    lu_solve(nd, o->mlu, o->piv, b);
    for (int i = 0; i < nd; ++i) out[(v * ne + e) * nd + i] = b[i];
  }
}

/* Residual of every element.  Elements are independent (each writes its own output and,
 * on storing steps, its own flux-buffer slots), so a build with OpenMP (-fopenmp, the
 * all-cores timing variant) splits them over threads, each with its own scratch; the
 * arithmetic of each element is the same in both builds, and so are the results. */
static void all_elements_rhs(adgref* o, const double* u, int stage, int mode, double* out) {
  size_t nsc = (size_t)o->nv * o->nd;
#pragma omp parallel
  {
    double* F = malloc(sizeof(double) * 5 * nsc);
    double* V = F + 3 * nsc;
    double* S = V + nsc;
#pragma omp for schedule(static)
    for (int64_t e = 0; e < o->ne; ++e) element_rhs(o, u, e, stage, mode, out, F, V, S);
    free(F);
  }
}

void adgref_rhs(adgref* o, const double* u, double* k) { all_elements_rhs(o, u, 0, 0, k); }

int adgref_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void adgref_rhs_elements(adgref* o, const double* u, const int64_t* elems, int64_t n_sel,
                         double* k) {
  /* writes k for the selected elements as [sel][var][node] */
  int64_t sz = adgref_state_size(o);
  double* tmp = o->kk;
  (void)sz;
  for (int64_t s = 0; s < n_sel; ++s) {
    int64_t e = elems[s];
    element_rhs(o, u, e, 0, 0, tmp, o->F, o->V, o->S);
    for (int v = 0; v < o->nv; ++v)
      for (int i = 0; i < o->nd; ++i)
        k[(s * o->nv + v) * o->nd + i] = tmp[(v * o->ne + e) * o->nd + i];
  }
}

static void stage_coeffs(adgref* o, int stage) {
  int maxk = (o->p.delay_mode == ADGREF_DELAY_RANDOM) ? o->p.random_delay_max : o->p.max_delay;
  if (maxk > 15) maxk = 15;
  for (int kt = 0; kt <= maxk; ++kt) adgref_at_coeffs(o->np, kt + o->rkc[stage], o->coef[kt]);
}

int adgref_step(adgref* o, int n_steps) {
  int64_t sz = adgref_state_size(o);
  double dt = o->p.dt;
  for (int it = 0; it < n_steps; ++it) {
    int64_t n = o->step;
    /* flag and delay counter at the start of step n (Algorithms 2 and 3) */
    if (o->p.delay_mode == ADGREF_DELAY_RANDOM) {
      for (int f = 0; f < o->niface; ++f)
        o->idelay[f] = random_delay(o->p.flux, o->np, o->p.seed, o->p.random_delay_max, n,
                                    o->niface, f);
      o->comm = 0;
    } else {
      int c;
      if (o->p.flux == ADGREF_FLUX_SYNC) c = 1;
      else if (o->p.flux == ADGREF_FLUX_STD) c = (n % o->p.max_delay) == 0;
      else c = (n % (o->p.max_delay + o->np + 1)) < (o->np + 1);
      o->comm = c;
      o->kcount = c ? 0 : o->kcount + 1;
    }
    if (!o->rk2n) {
      /* two-register scheme, Eq. 10 */
      memcpy(o->r, o->w, sizeof(double) * sz);
      for (int m = 0; m < o->stages; ++m) {
        stage_coeffs(o, m);
        all_elements_rhs(o, o->r, m, 1, o->kk);
        for (int64_t i = 0; i < sz; ++i) {
          if (m + 1 < o->stages) o->r[i] = o->w[i] + dt * o->rka[m] * o->kk[i];
          o->w[i] = o->w[i] + dt * o->rkb[m] * o->kk[i];
        }
      }
    } else {
      /* 2N scheme: q <- A_m q + dt k_m ; w <- w + B_m q */
      for (int m = 0; m < o->stages; ++m) {
        stage_coeffs(o, m);
        all_elements_rhs(o, o->w, m, 1, o->kk);
        for (int64_t i = 0; i < sz; ++i) {
          o->q[i] = (m == 0 ? 0.0 : o->rka[m] * o->q[i]) + dt * o->kk[i];
          o->w[i] = o->w[i] + o->rkb[m] * o->q[i];
        }
      }
    }
    o->step += 1;
    o->t += dt;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Diagnostics: conserved totals, initial conditions, L2 error, time step.               */
/* ------------------------------------------------------------------------------------ */
void adgref_conservation(const adgref* o, const double* u, double* sums) {
  for (int v = 0; v < o->nv; ++v) {
    double s = 0.0;
    for (int64_t e = 0; e < o->ne; ++e)
      for (int q = 0; q < o->nd; ++q) s += o->wq[q] * u[(v * o->ne + e) * o->nd + q];
    sums[v] = s;
  }
}

static void node_position(const adgref* o, int64_t e, const double* xi, double* x) {
  int c[3];
  elem_coords(o, e, c);
  for (int d = 0; d < o->dim; ++d) x[d] = o->p.lo[d] + (c[d] + 0.5 * (xi[d] + 1.0)) * o->h[d];
}

/* Isentropic vortex of the 2D benchmark (exact solution below Eq. 16's test-case text),  */
/* on the periodic box: the centre is advected with speed (1, 0) and the nearest periodic */
/* image is used.  In 3D the same vortex is extruded along z.                             */
static void vortex_exact(const adgref* o, const double* x, double t, double beta, double x0,
                         double y0, double* w) {
  const double pi = 3.14159265358979323846;
  double g = o->p.gamma;
  double Lx = o->p.hi[0] - o->p.lo[0], Ly = o->p.hi[1] - o->p.lo[1];
  double dx = x[0] - (x0 + t);
  double dy = x[1] - y0;
  dx -= Lx * floor(dx / Lx + 0.5);
  dy -= Ly * floor(dy / Ly + 0.5);
  double r2 = dx * dx + dy * dy;
  double ex = exp(1.0 - r2);
  double u = 1.0 - beta * ex * dy / (2.0 * pi);
  double v = beta * ex * dx / (2.0 * pi);
  double rho = pow(1.0 - (g - 1.0) / (16.0 * g * pi * pi) * beta * beta * ex * ex, 1.0 / (g - 1.0));
  double p = pow(rho, g);
  w[0] = rho;
  w[1] = rho * u;
  w[2] = rho * v;
  if (o->dim == 3) w[3] = 0.0;
  w[o->dim + 1] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

void adgref_init_vortex(const adgref* o, double* u, double t, double beta, double x0, double y0) {
  for (int64_t e = 0; e < o->ne; ++e)
    for (int q = 0; q < o->nd; ++q) {
      double xi[3], x[3], w[5];
      int idx[3];
      vol_point(o, q, xi, idx);
      node_position(o, e, xi, x);
      vortex_exact(o, x, t, beta, x0, y0, w);
      for (int v = 0; v < o->nv; ++v) u[(v * o->ne + e) * o->nd + q] = w[v];
    }
}

/* Taylor-Green vortex (3D periodic [0,2pi]^3 case), rho0 = V0 = 1, p0 = 1/(gamma M^2). */
void adgref_init_tgv(const adgref* o, double* u, double mach) {
  double g = o->p.gamma;
  double p0 = 1.0 / (g * mach * mach);
  for (int64_t e = 0; e < o->ne; ++e)
    for (int q = 0; q < o->nd; ++q) {
      double xi[3], x[3] = {0, 0, 0};
      int idx[3];
      vol_point(o, q, xi, idx);
      node_position(o, e, xi, x);
      double ux = sin(x[0]) * cos(x[1]) * cos(x[2]);
      double uy = -cos(x[0]) * sin(x[1]) * cos(x[2]);
      double uz = 0.0;
      double p = p0 + (cos(2.0 * x[0]) + cos(2.0 * x[1])) * (cos(2.0 * x[2]) + 2.0) / 16.0;
      double rho = p / p0;
      double w[5] = {rho, rho * ux, rho * uy, rho * uz, 0.0};
      w[4] = p / (g - 1.0) + 0.5 * rho * (ux * ux + uy * uy + uz * uz);
      for (int v = 0; v < o->nv; ++v) u[(v * o->ne + e) * o->nd + q] = w[v];
    }
}

/* Absolute L2 errors (density, momentum vector, energy) against the exact vortex, with */
/* (p+2)^d Gauss points per element and the discrete solution interpolated there.      */
void adgref_l2_error_vortex(const adgref* o, const double* u, double t, double beta, double x0,
                            double y0, double* err3) {
  int m = o->nn + 1;
  double xg[MAXN + 1], wg[MAXN + 1];
  adgref_gauss(m, xg, wg);
  double J = 1.0;
  for (int d = 0; d < o->dim; ++d) J *= o->h[d] / 2.0;
  int npts = 1;
  for (int d = 0; d < o->dim; ++d) npts *= m;
  double acc[3] = {0, 0, 0};
  for (int64_t e = 0; e < o->ne; ++e)
    for (int pt = 0; pt < npts; ++pt) {
      double xi[3], x[3], wt = J, wex[5], wh[5];
      int t2 = pt;
      for (int d = 0; d < o->dim; ++d) {
        xi[d] = xg[t2 % m];
        wt *= wg[t2 % m];
        t2 /= m;
      }
      node_position(o, e, xi, x);
      vortex_exact(o, x, t, beta, x0, y0, wex);
      for (int v = 0; v < o->nv; ++v) {
        double s = 0.0;
        for (int j = 0; j < o->nd; ++j) s += u[(v * o->ne + e) * o->nd + j] * basis_at(o, j, xi);
        wh[v] = s;
      }
      double dr = wh[0] - wex[0], de = wh[o->dim + 1] - wex[o->dim + 1], dm = 0.0;
      for (int d = 0; d < o->dim; ++d) dm += (wh[1 + d] - wex[1 + d]) * (wh[1 + d] - wex[1 + d]);
      acc[0] += wt * dr * dr;
      acc[1] += wt * dm;
      acc[2] += wt * de * de;
    }
  for (int i = 0; i < 3; ++i) err3[i] = sqrt(acc[i]);
}

/* Time step from a CFL number: dt = cfl h_min / ((2p+1) max(|u| + c)), then shortened so */
/* that a whole number of steps reaches t_end (if t_end > 0).                             */
double adgref_dt_from_cfl(const adgref* o, const double* u, double cfl, double t_end) {
  double smax = 0.0;
  for (int64_t e = 0; e < o->ne; ++e)
    for (int q = 0; q < o->nd; ++q) {
      double w[5];
      for (int v = 0; v < o->nv; ++v) w[v] = u[(v * o->ne + e) * o->nd + q];
      double rho = w[0], u2 = 0.0, kin = 0.0;
      for (int d = 0; d < o->dim; ++d) {
        double ud = w[1 + d] / rho;
        u2 += ud * ud;
        kin += w[1 + d] * ud;
      }
      double p = (o->p.gamma - 1.0) * (w[o->dim + 1] - 0.5 * kin);
      double s = sqrt(u2) + sqrt(o->p.gamma * p / rho);
      if (s > smax) smax = s;
    }
  double hmin = o->h[0];
  for (int d = 1; d < o->dim; ++d)
    if (o->h[d] < hmin) hmin = o->h[d];
  double dt = cfl * hmin / ((2.0 * o->p.degree + 1.0) * smax);
  if (t_end > 0.0) {
    double nsteps = ceil(t_end / dt);
    dt = t_end / nsteps;
  }
  return dt;
}

void adgref_info(const adgref* o, int64_t* step, double* t, double* dt) {
  if (step) *step = o->step;
  if (t) *t = o->t;
  if (dt) *dt = o->p.dt;
}
