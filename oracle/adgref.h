/*
 * adgref: plain, slow FP64 CPU oracle of the asynchronous discontinuous Galerkin (ADG)
 * method for the compressible Euler equations (arXiv 2603.28710).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or call this
 * code; only the test suite, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every quantity is computed by its plain definition: dense element quadrature on the
 * weak form (Eq. 6), a dense mass matrix solved by Gaussian elimination (Eq. 7), the
 * Rusanov flux with the paper's dissipation parameter (Eq. 8-9), the two-register
 * low-storage Runge-Kutta update (Eq. 10), the delayed flux (Eq. 13), the AT flux from
 * the moment constraints (Eq. 14-15) and the communication-avoiding schedules
 * (Algorithms 2 and 3).  Compiled with -O2 -ffp-contract=off and no fast-math.
 */
#ifndef ADGREF_H
#define ADGREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ADGREF_FLUX_SYNC = 0, ADGREF_FLUX_STD = 1, ADGREF_FLUX_AT = 2, ADGREF_FLUX_AT_TRACE = 3 };
enum { ADGREF_DELAY_CAA = 0, ADGREF_DELAY_RANDOM = 1 };
enum { ADGREF_RK22 = 0, ADGREF_RK33 = 1, ADGREF_CK45 = 2 };

typedef struct {
  int dim;            /* 2 or 3 */
  int n_elem[3];      /* elements per direction (periodic, uniform) */
  double lo[3], hi[3];
  int degree;         /* polynomial degree N_p of the DG basis */
  int P[3];           /* logical subdomains (processing elements) per direction */
  int max_delay;      /* L of Algorithms 2 and 3 */
  int flux;           /* ADGREF_FLUX_* */
  int rk;             /* ADGREF_RK* */
  int delay_mode;     /* ADGREF_DELAY_* */
  int random_delay_max;
  int at_np;          /* AT stencil: N_p + 1 stored levels; <= 0 means N_p = degree */
  uint64_t seed;
  double gamma;
  double dt;
} adgref_params;

typedef struct adgref adgref;

/* ---- building blocks (each pinned by the test suite) ---- */
int adgref_gauss(int n, double* x, double* w);
double adgref_lagrange(int n, const double* x, int a, double xi);
double adgref_lagrange_deriv(int n, const double* x, int a, double xi);
int adgref_at_coeffs(int np, double km, double* c);
int adgref_rk_tableau(int scheme, double* a, double* b, double* c, double* butcher_a, double* butcher_b);
void adgref_euler_flux(int dim, double gamma, const double* w, int dir, double* f);
void adgref_llf(int dim, double gamma, const double* wm, const double* wp, const double* normal,
                double* fhat);
uint64_t adgref_splitmix64(uint64_t x);
int adgref_schedule(int flux, int delay_mode, int max_delay, int np, const int* P, int dim,
                    uint64_t seed, int dmax, int64_t n0, int count, int32_t* comm, int32_t* k,
                    int32_t* iface_delay);
int adgref_num_interfaces(int dim, const int* P);

/* ---- solver ---- */
adgref* adgref_create(const adgref_params* prm);
void adgref_destroy(adgref* o);
int64_t adgref_state_size(const adgref* o);
void adgref_set_state(adgref* o, const double* u);
void adgref_get_state(const adgref* o, double* u);
int adgref_step(adgref* o, int n_steps);
void adgref_rhs(adgref* o, const double* u, double* k);
/* Threads the element loops of adgref_rhs and adgref_step use: 1, or the OpenMP thread
 * count in the all-cores build (compiled with -fopenmp; same results). */
int adgref_threads(void);
void adgref_rhs_elements(adgref* o, const double* u, const int64_t* elems, int64_t n_sel,
                         double* k);
void adgref_conservation(const adgref* o, const double* u, double* sums);
void adgref_init_vortex(const adgref* o, double* u, double t, double beta, double x0, double y0);
void adgref_init_tgv(const adgref* o, double* u, double mach);
void adgref_l2_error_vortex(const adgref* o, const double* u, double t, double beta, double x0,
                            double y0, double* err3);
double adgref_dt_from_cfl(const adgref* o, const double* u, double cfl, double t_end);
void adgref_info(const adgref* o, int64_t* step, double* t, double* dt);

#ifdef __cplusplus
}
#endif
#endif
