/*
 * rcp_oracle.h -- plain, slow FP64 CPU oracle for the Adam-based
 * Clarke-Wiley inflation protocol (random close packing of polydisperse
 * spheres, arxiv 2608.12235).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include,
 * link, load or call this code: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no code, header,
 * constant or helper with the CUDA library; the two are compared element
 * by element on the same seeded inputs.
 *
 * Every function states the passage of the paper it follows.  Where the
 * paper is silent, the reading taken is stated beside the code (they are
 * collected under "Readings" in the design notes of the repository).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -ffast-math):
 * every floating-point operation is an IEEE-754 binary64 operation in the
 * order written, so results are reproducible bit for bit.
 */
#ifndef RCP_ORACLE_H
#define RCP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- schedule and optimiser parameters (the oracle's own copy) ---- */
typedef struct {
    int    d;            /* spatial dimension: 2 or 3 */
    double L[3];         /* periodic box edges */
    double phi0;         /* initial packing fraction (sets kappa_0) */
    double eps;          /* overlap stiffness epsilon of Eq. energy */
    double beta1, beta2, adam_eps;   /* Adam (Kingma-Ba) */
    double skin_s;       /* size-proportional skin fraction s */
    double skin_theta;   /* rebuild threshold theta, in (0,1) */
    double skin_abs;     /* absolute skin sigma0 = skin_abs * eta_x,0 */
    double lr_x;         /* position lr, in units of kappa * D_ref */
    double lr_kappa;     /* kappa lr, in units of kappa */
    double delta_star0;  /* target mean overlap of the first rung */
    double tol;          /* stopping tolerance on max fractional overlap */
    int    Y, X;         /* Eq. trigger */
    long   n_min;        /* minimum rung budget */
    int    n_down;       /* number of rungs after the first (mu / 10 each) */
    int    n_cycles;     /* mu cycles after the descent */
    long   max_iters;    /* safety cap on the total iteration count */
    double kappa_init;   /* > 0: start the run at this kappa instead of kappa_0
                            (sigma0 is still that of kappa_0); 0: kappa_0 */
    int    walls;        /* bit a set: flat hard walls at 0 and L_a bound axis a
                            (no minimum image, no wrap); 0: periodic box */
    int    container;    /* curved wall: 0 none, 1 ball (disk when d = 2), 2 cylinder
                            about z; radius min L_a/2 over its axes, box centre */
} orc_params;

typedef struct {
    long   iters;        /* Adam steps taken */
    long   rebuilds;     /* neighbour-list builds */
    int    stopped;      /* 1 if the stopping criterion fired */
    double kappa;        /* kappa at stop */
    double max_delta;    /* max fractional overlap at stop */
    double energy;       /* E at stop (with the final rung's mu = 0) */
    double kappa_c;      /* shrink-to-contact kappa */
    double phi;          /* shrink-to-contact packing fraction */
} orc_result;

/* Frozen spheres (stages of the sequential cascade, Sec. IV): wherever a
 * function takes D0, an entry D0[i] < 0 marks sphere i as frozen, with fixed
 * contact diameter -D0[i] and a position that the run does not move. */

/* Flat hard walls: the wall mask in force for every geometric function
 * below (bit a: axis a bounded by walls at 0 and L_a).  orc_run uses its
 * parameter's mask for the run. */
void   orc_set_walls(int mask);
int    orc_get_walls(void);
void   orc_set_container(int type);   /* 0 none, 1 ball / disk, 2 cylinder about z */
int    orc_get_container(void);

/* Threads of the row loop of the evaluation and of the Adam step (OpenMP;
 * 1 by default).  Results do not depend on it: rows are independent and
 * every global sum keeps its fixed tree. */
void   orc_set_threads(int n);
int    orc_get_threads(void);

/* ---- input-side primitives ---- */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k);
void   orc_init_positions(uint64_t seed, long n, int d, const double* L, double* x);
int    orc_place(uint64_t seed, long n, int d, const double* L, const double* D0, double kappa,
                 int max_rounds, double* x, int* round_of);
double orc_tree_sum(const double* a, long n);
double orc_cbrt(double a);
void   orc_moments(const double* D0, long n, double out[3]); /* sum D, D^3, D^4 */
double orc_kappa0(const double* D0, long n, int d, const double* L, double phi0);
double orc_n_trig(long n, int d, int Y, int X);

/* ---- neighbour structure ---- */
double orc_rho(double D0, double kappa_b, double s, double sigma0);
int    orc_levels(const double* D0, long n, double kappa_b, double s, double sigma0,
                  int* lvl, double* rho_max_lvl /* [32] */);
long   orc_grid_n(double L, long count, double V, double occ);
void   orc_cell_keys(const double* x, const double* D0, long n, int d, const double* L,
                     double kappa_b, double s, double sigma0, double occ, uint64_t* key);
int    orc_listed(const double* xi, const double* xj, int d, const double* L,
                  double rho_i, double rho_j);
long   orc_list_brute(const double* x, const double* D0, long n, int d, const double* L,
                      double kappa_b, double s, double sigma0,
                      long* rowptr, int* col, long cap);
long   orc_list_grid(const double* x, const double* D0, long n, int d, const double* L,
                     double kappa_b, double s, double sigma0,
                     long* rowptr, int* col, long cap);
long   orc_list_grid_occ(const double* x, const double* D0, long n, int d, const double* L,
                         double kappa_b, double s, double sigma0, double occ,
                         long* rowptr, int* col, long cap);
long   orc_row_brute(const double* x, const double* D0, long n, int d, const double* L,
                     double kappa_b, double s, double sigma0, long i, int* col, long cap);

/* ---- Eq. energy and its gradient ---- */
void   orc_energy_grad_brute(const double* x, const double* D0, long n, int d, const double* L,
                             double kappa, double mu, double eps,
                             double* E, double* g, double* dEdk, double* maxdelta);
void   orc_energy_grad_list(const double* x, const double* D0, long n, int d, const double* L,
                            double kappa, double mu, double eps,
                            const long* rowptr, const int* col,
                            double* E, double* g, double* dEdk, double* maxdelta);
void   orc_row_grad(const double* x, const double* D0, long n, int d, const double* L,
                    double kappa, double eps, long i, double* g_i, double* e_i,
                    double* k_i, double* maxd_i);

/* ---- Adam (applied jointly to the coordinates and kappa) ---- */
void   orc_adam_update(double* p, double* m, double* v, const double* g, long n,
                       double eta, double beta1, double beta2, double adam_eps,
                       double b1, double b2);
double orc_wrap(double x, double L);

/* ---- shrink to contact and packing fraction ---- */
double orc_shrink_kappa(const double* x, const double* D0, long n, int d, const double* L,
                        double kappa, const long* rowptr, const int* col);
double orc_phi(const double* D0, long n, int d, const double* L, double kappa);

/* ---- the whole protocol ---- */
void   orc_params_default(orc_params* p);
int    orc_run(const orc_params* p, const double* D0, long n, uint64_t seed,
               double* x_io, int x_given, orc_result* res, double* trace, long trace_cap);

long   orc_sample_iterations(const orc_params* p, const double* D0, long n, double* x, double kappa,
                             double mu, double eta_x, double eta_k, double sigma0, long iters);

#ifdef __cplusplus
}
#endif
#endif
