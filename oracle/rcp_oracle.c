/*
 * rcp_oracle.c -- plain FP64 CPU oracle of the Adam-based inflation protocol
 * (arxiv 2608.12235, Appendix A).  TEST INFRASTRUCTURE ONLY: the product
 * path never includes, links or calls this file.
 *
 * What is the paper's and what is a reading:
 *   - Eq. energy (App. A): E = eps/2 sum_{i<j} (1 - r_ij/d_ij)^2 Theta(1 - r_ij/d_ij)
 *     - mu sum_i D_i, d_ij = (D_i + D_j)/2, D_i = kappa D_i^0.  The paper's.
 *   - Theta(0) = 0 (a pair counts only when the overlap is strictly positive),
 *     eps = 1: readings.
 *   - the gradients w.r.t. x_i and kappa: derived from Eq. energy here; the
 *     paper prints none.  A pair with r_ij = 0 contributes its energy and its
 *     kappa-derivative but no position gradient (subgradient reading).
 *   - Adam on the coordinates and kappa (App. A) with the Kingma-Ba update and
 *     its default constants: the paper names Adam but not its constants.
 *   - the rung schedule built on Eq. trigger (App. A); rung values of mu and of
 *     the learning rate are readings (the paper leaves them to its code).
 *   - stop when the largest fractional overlap 1 - r/d is below 5e-4 (App. A),
 *     then shrink kappa uniformly until the last overlap vanishes and report
 *     the solid-volume fraction (Sec. II, App. A).
 *   - summation order: every global sum is a pairwise tree over the particle
 *     index, zero-padded to a power of two; every per-particle sum is a left
 *     fold over the partners in ascending index.  This is a reading that makes
 *     the FP64 result reproducible; the paper's threaded code is not (Data and
 *     code availability).
 *   - the neighbour structure (size-stratified cell levels with a skin) is the
 *     implementation's, not the paper's k-d tree (App. A); the energy and the
 *     gradient never depend on it, because a pair that is listed but does not
 *     overlap contributes exactly nothing.
 *   - frozen spheres, for the stages of the sequential cascade (Sec. IV: a
 *     finer class is seated into the voids of the coarser ones and inflated
 *     to contact while those are held fixed): an entry D0[i] < 0 marks sphere
 *     i as frozen, with contact diameter -D0[i] that kappa does not scale and
 *     a position that Adam does not move.  Its coordinates are constants of
 *     the energy, not variables: their gradient is zero.  The growth term and
 *     the moments that scale the schedule sum over the mobile spheres only.
 *     The whole encoding is a reading; the paper describes the protocol, not
 *     its arithmetic.
 *   - flat hard walls (Sec. II: each axis periodic or bounded by a wall):
 *     axis a with bit a of the wall mask set has walls at 0 and L_a; it takes
 *     no minimum image and no wrap.  A sphere meets a wall when the distance
 *     h from its centre to the wall is below its contact radius rad = kappa
 *     D^0 / 2 (F/2 frozen); delta = 1 - h/rad is the pair rule against its
 *     mirror image, and the term eps/2 delta^2 joins its row after the pair
 *     fold (axes in order, the wall at 0 before the wall at L_a).  Readings.
 *   - curved hard walls (Sec. II, Fig. 2: circular, cylindrical and spherical
 *     domains): a container of radius R = min over its axes of L_a/2 about the
 *     box centre -- a ball over every axis (a disk when d = 2) or a cylinder
 *     about the z axis (circle in x, y).  Its axes are bounded (no minimum
 *     image, no wrap); h = R - |x - c| over them, delta = 1 - h/rad as for a
 *     flat wall, the term after the flat walls'; kappa_0 and phi take the
 *     container's volume.  Readings.
 */
#include "rcp_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Threads for the row loop of orc_energy_grad_list and the coordinate loop
 * of the Adam step (OpenMP; 1 unless orc_set_threads asks for more).  Each
 * row's fold and each coordinate's update are independent and every global
 * sum keeps its fixed tree over the particle index, so no result depends on
 * the thread count. */
static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

#define ORC_PI 3.141592653589793
#define ORC_KMAX 32
#define ORC_NMAX (1L << 19)

/* Wall mask of the boundary in force (bit a: flat walls bound axis a).  A
 * module setting rather than an argument of every geometric function;
 * orc_run sets it from its parameters for the run and restores it. */
static int g_walls = 0;

void orc_set_walls(int mask) { g_walls = mask; }
int orc_get_walls(void) { return g_walls; }

/* Curved container (0 none, 1 ball over every axis / disk when d = 2,
 * 2 cylinder about z), a module setting like the wall mask. */
static int g_container = 0;

void orc_set_container(int type) { g_container = type; }
int orc_get_container(void) { return g_container; }

/* Axis a lies in the container's cross-section. */
static int in_container(int a, int d) { return g_container == 1 ? a < d : (g_container == 2 ? a < 2 : 0); }

/* Bounded axis: flat walls or the container; no minimum image, no wrap. */
static int walled(int a) { return ((g_walls >> a) & 1) || in_container(a, 3); }

/* Flat wall terms only on the axes of the wall mask. */
static int flat_wall(int a) { return (g_walls >> a) & 1; }

/* Container radius: half the smallest box edge over its axes. */
static double container_R(int d, const double* L)
{
    double R = INFINITY;
    for (int a = 0; a < d; ++a)
        if (in_container(a, d) && 0.5 * L[a] < R) R = 0.5 * L[a];
    return R;
}

/* Distance from x to the container's axis or centre over its axes, and the
 * offsets x_a - L_a/2. */
static double container_dist(const double* x, int d, const double* L, double* off)
{
    double s2 = 0.0;
    for (int a = 0; a < d; ++a) {
        off[a] = in_container(a, d) ? x[a] - 0.5 * L[a] : 0.0;
        s2 = s2 + off[a] * off[a];
    }
    return sqrt(s2);
}

/* Contact diameter of a sphere at scale kappa: kappa D^0 for a mobile sphere,
 * the fixed -D0 for a frozen one (D0 < 0). */
static double size_at(double D0, double kappa) { return D0 >= 0.0 ? kappa * D0 : -D0; }

/* The part of D0 that kappa scales: D0 for a mobile sphere, 0 for a frozen one. */
static double mobile_part(double D0) { return D0 > 0.0 ? D0 : 0.0; }

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's reference form): the
 * generator's state advances by the golden-ratio increment and each output is
 * the state passed through the variant-13 mixer.  Output k (0-based) of the
 * stream seeded with `seed` is therefore mix(seed + (k+1) * gamma). */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Wrap a coordinate back into [0, L) after a step shorter than L. */
double orc_wrap(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

/* Initial configuration (reading of "positions uniform random at the initial
 * packing fraction"; the paper places a dilute non-overlapping configuration,
 * App. A): coordinate a of particle i is L_a * u with u the top 53 bits of
 * SplitMix64 output number d*i + a, scaled by 2^-53. */
void orc_init_positions(uint64_t seed, long n, int d, const double* L, double* x)
{
    for (long i = 0; i < n; ++i)
        for (int a = 0; a < d; ++a) {
            uint64_t z = orc_splitmix64_at(seed, (uint64_t)(d * i + a));
            double u = (double)(z >> 11) * 0x1.0p-53;
            x[d * i + a] = orc_wrap(L[a] * u, L[a]);
        }
}

/* Non-overlapping placement (App. A starts from a dilute configuration with
 * no overlaps, built with cell lists; the paper gives no further detail).  Reading: random sequential addition by size class,
 * largest class first, each class in rounds.  With rho_i = (kappa D_i^0) / 2
 * the class is k_i = max{k in [0, 31] : rho_i 2^k <= max rho} (the neighbour
 * structure's rule with no skin).  In round a of class k every sphere of the
 * class not yet placed draws candidate a from SplitMix64 outputs
 * d (a n + i) + c (axis c), so every first draw is the uniform initial state
 * of orc_init_positions.  A candidate is kept unless it overlaps a sphere
 * already placed (any earlier class or round) or the candidate of a sphere of
 * the class that precedes it (larger D^0, then lower index).  Overlap:
 * r_ij^2 < (rho_i + rho_j)^2, minimum image.  Brute force: every candidate is
 * tested against every sphere.  attempt[i] (optional) receives the round in
 * which sphere i was placed.  Returns the largest number of rounds a class
 * took, or -1 if a class still has spheres unplaced after max_rounds (those
 * keep their last candidates).  With flat walls a candidate is also rejected
 * when it meets one (distance to the wall below rho_i).  Frozen spheres (D0 < 0) count as placed from
 * the start, at the positions x holds on entry; they never draw. */
int orc_place(uint64_t seed, long n, int d, const double* L, const double* D0, double kappa, int max_rounds,
              double* x, int* attempt)
{
    char* placed = (char*)calloc((size_t)n, 1);
    for (long i = 0; i < n; ++i) placed[i] = D0[i] < 0.0;
    char* keep = (char*)malloc((size_t)n);
    int* cls = (int*)malloc(sizeof(int) * (size_t)n);
    double* rad = (double*)malloc(sizeof(double) * (size_t)n);
    double* cand = (double*)malloc(sizeof(double) * (size_t)(n * d));
    orc_init_positions(seed, n, d, L, cand);   /* every sphere's first draw */
    double rmax = 0.0;
    for (long i = 0; i < n; ++i) {
        rad[i] = orc_rho(D0[i], kappa, 0.0, 0.0);
        if (rad[i] > rmax) rmax = rad[i];
    }
    int kmax = 0;
    for (long i = 0; i < n; ++i) {
        int k = 0;
        while (k + 1 < ORC_KMAX && ldexp(rad[i], k + 1) <= rmax) ++k;
        cls[i] = k;
        if (k > kmax) kmax = k;
    }
    int worst = 0, failed = 0;
    for (int k = 0; k <= kmax && !failed; ++k) {
        long left = 0;
        for (long i = 0; i < n; ++i) left += cls[i] == k && !placed[i];
        int r = 0;
        for (; r < max_rounds && left > 0; ++r) {
            for (long i = 0; i < n; ++i) {
                if (cls[i] != k || placed[i]) continue;
                for (int a = 0; a < d; ++a) {
                    uint64_t z = orc_splitmix64_at(seed, (uint64_t)d * ((uint64_t)r * (uint64_t)n + (uint64_t)i) +
                                                             (uint64_t)a);
                    double u = (double)(z >> 11) * 0x1.0p-53;
                    cand[d * i + a] = orc_wrap(L[a] * u, L[a]);
                }
            }
            for (long i = 0; i < n; ++i) {
                if (cls[i] != k || placed[i]) continue;
                keep[i] = 1;
                for (int a = 0; a < d; ++a)   /* a candidate must not meet a wall either */
                    if (flat_wall(a) && (cand[d * i + a] < rad[i] || L[a] - cand[d * i + a] < rad[i])) keep[i] = 0;
                if (g_container) {
                    double off[3];
                    if (container_R(d, L) - container_dist(&cand[d * i], d, L, off) < rad[i]) keep[i] = 0;
                }
                for (long j = 0; j < n && keep[i]; ++j) {
                    if (j == i) continue;
                    if (placed[j]) {
                        if (orc_listed(&cand[d * i], &x[d * j], d, L, rad[i], rad[j])) keep[i] = 0;
                    } else if (cls[j] == k && (D0[j] > D0[i] || (D0[j] == D0[i] && j < i))) {
                        if (orc_listed(&cand[d * i], &cand[d * j], d, L, rad[i], rad[j])) keep[i] = 0;
                    }
                }
            }
            for (long i = 0; i < n; ++i) {
                if (cls[i] != k || placed[i] || !keep[i]) continue;
                for (int a = 0; a < d; ++a) x[d * i + a] = cand[d * i + a];
                placed[i] = 1;
                if (attempt) attempt[i] = r;
                --left;
            }
        }
        if (r > worst) worst = r;
        if (left > 0) failed = 1;
    }
    for (long i = 0; i < n; ++i)
        if (!placed[i]) {
            if (attempt) attempt[i] = -1;
            for (int a = 0; a < d; ++a) x[d * i + a] = cand[d * i + a];
        } else if (D0[i] < 0.0 && attempt) {
            attempt[i] = 0;
        }
    free(placed);
    free(keep);
    free(cls);
    free(rad);
    free(cand);
    return failed ? -1 : worst;
}

/* Pairwise tree sum: sum(a[0:m]) = sum(a[0:m/2]) + sum(a[m/2:m]) with m the
 * smallest power of two >= n and a[i] = 0 for i >= n. */
static double tree_rec(const double* a, long lo, long len, long n)
{
    if (len == 1) return lo < n ? a[lo] : 0.0;
    long h = len / 2;
    double s0 = tree_rec(a, lo, h, n);
    double s1 = tree_rec(a, lo + h, h, n);
    return s0 + s1;
}

double orc_tree_sum(const double* a, long n)
{
    long m = 1;
    while (m < n) m *= 2;
    return tree_rec(a, 0, m, n);
}

/* Cube root by a fixed count of Newton steps y <- (2y + a/y^2)/3 from y = 1:
 * every step is a correctly rounded IEEE operation, so any conforming machine
 * gets the same bits (libm cbrt is not correctly rounded). */
double orc_cbrt(double a)
{
    if (!(a > 0.0)) return 0.0;
    double y = 1.0;
    for (int it = 0; it < 200; ++it) y = (2.0 * y + a / (y * y)) / 3.0;
    return y;
}

/* out[0] = sum D, out[1] = sum D^3, out[2] = sum D^4 (tree sums) over the
 * mobile spheres (a frozen sphere's term is 0). */
void orc_moments(const double* D0, long n, double out[3])
{
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) t[i] = mobile_part(D0[i]);
    out[0] = orc_tree_sum(t, n);
    for (long i = 0; i < n; ++i) { double D = mobile_part(D0[i]); t[i] = (D * D) * D; }
    out[1] = orc_tree_sum(t, n);
    for (long i = 0; i < n; ++i) { double D = mobile_part(D0[i]); t[i] = (D * D) * (D * D); }
    out[2] = orc_tree_sum(t, n);
    free(t);
}

static double box_volume(int d, const double* L)
{
    return d == 2 ? L[0] * L[1] : (L[0] * L[1]) * L[2];
}

/* Volume (area when d = 2) the spheres fill: the container's, else the box's. */
static double solid_volume(int d, const double* L)
{
    double R = container_R(d, L);
    if (g_container == 1) return d == 2 ? (ORC_PI * R) * R : (((4.0 / 3.0) * ORC_PI) * ((R * R) * R));
    if (g_container == 2) return ((ORC_PI * R) * R) * L[2];
    return box_volume(d, L);
}

/* kappa such that the solid-volume fraction of {kappa D_i^0} equals phi0
 * (mobile spheres only: a frozen sphere's term is 0). */
double orc_kappa0(const double* D0, long n, int d, const double* L, double phi0)
{
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double V = solid_volume(d, L), k;
    if (d == 2) {
        for (long i = 0; i < n; ++i) { double D = mobile_part(D0[i]); t[i] = D * D; }
        k = sqrt((phi0 * V) / ((ORC_PI / 4.0) * orc_tree_sum(t, n)));
    } else {
        for (long i = 0; i < n; ++i) { double D = mobile_part(D0[i]); t[i] = (D * D) * D; }
        k = orc_cbrt((phi0 * V) / ((ORC_PI / 6.0) * orc_tree_sum(t, n)));
    }
    free(t);
    return k;
}

/* Eq. trigger (App. A): n_trig = 4000 Y + X sqrt(N d) - 2000. */
double orc_n_trig(long n, int d, int Y, int X)
{
    return (4000.0 * (double)Y + (double)X * sqrt((double)(n * (long)d))) - 2000.0;
}

/* ------------------------------------------------------------------------ */
/* Neighbour structure.  Interaction radius of particle i at build time:
 * rho_i = kappa_b D_i^0 (1/2 + s) + sigma0, i.e. half its diameter plus its
 * skin sigma_i = s kappa_b D_i^0 + sigma0.  A pair is listed iff its
 * minimum-image distance is below rho_i + rho_j = kappa_b d_ij^0 + sigma_i +
 * sigma_j.  A frozen sphere has its fixed diameter in place of kappa_b D_i^0. */
double orc_rho(double D0, double kappa_b, double s, double sigma0)
{
    return size_at(D0, kappa_b) * (0.5 + s) + sigma0;
}

/* Minimum-image displacement x_i - x_j on every periodic axis (the plain
 * difference on a walled one), squared distance accumulated left to right. */
static double min_image(const double* xi, const double* xj, int d, const double* L, double* dx)
{
    double r2 = 0.0;
    for (int a = 0; a < d; ++a) {
        double t = xi[a] - xj[a];
        double h = 0.5 * L[a];
        if (walled(a)) { /* bounded axis: the plain difference */ }
        else if (t > h) t = t - L[a];
        else if (t < -h) t = t + L[a];
        dx[a] = t;
        r2 = r2 + t * t;
    }
    return r2;
}

int orc_listed(const double* xi, const double* xj, int d, const double* L,
               double rho_i, double rho_j)
{
    double dx[3];
    double r2 = min_image(xi, xj, d, L, dx);
    double c = rho_i + rho_j;
    return r2 < c * c;
}

/* Size classes: k_i = max{k in [0, 31] : rho_i 2^k <= max_j rho_j}. */
int orc_levels(const double* D0, long n, double kappa_b, double s, double sigma0,
               int* lvl, double* rho_max_lvl)
{
    double rmax = 0.0;
    for (long i = 0; i < n; ++i) {
        double r = orc_rho(D0[i], kappa_b, s, sigma0);
        if (r > rmax) rmax = r;
    }
    for (int k = 0; k < ORC_KMAX; ++k) rho_max_lvl[k] = 0.0;
    int nlev = 0;
    for (long i = 0; i < n; ++i) {
        double r = orc_rho(D0[i], kappa_b, s, sigma0);
        int k = 0;
        while (k + 1 < ORC_KMAX && ldexp(r, k + 1) <= rmax) ++k;
        lvl[i] = k;
        if (r > rho_max_lvl[k]) rho_max_lvl[k] = r;
        if (k + 1 > nlev) nlev = k + 1;
    }
    return nlev;
}

/* Cells per axis at a level: the largest power of two n <= 2^19 whose cell
 * volume holds at least `occ` spheres of the level on average,
 * h^3 count >= occ V with h = L/n (V the box volume, count the level's size).
 * The search scans every cell within the search radius, so any cell size is
 * correct; this one balances cell lookups against candidates. */
long orc_grid_n(double L, long count, double V, double occ)
{
    long n = 1;
    for (;;) {
        if (n >= ORC_NMAX) break;
        double h = L / (double)(2 * n);
        if (!(((h * h) * h) * (double)count >= occ * V)) break;
        n *= 2;
    }
    return n;
}

static long cell_of(double x, double L, long n)
{
    long c = (long)floor((x / L) * (double)n);
    if (c < 0) c = 0;
    if (c > n - 1) c = n - 1;
    return c;
}

/* Cell key: class in bits 57-61, then z, y, x cell indices of 19 bits each. */
static uint64_t pack_key(int k, long cz, long cy, long cx)
{
    return ((uint64_t)k << 57) | ((uint64_t)cz << 38) | ((uint64_t)cy << 19) | (uint64_t)cx;
}

void orc_cell_keys(const double* x, const double* D0, long n, int d, const double* L,
                   double kappa_b, double s, double sigma0, double occ, uint64_t* key)
{
    int* lvl = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double rml[ORC_KMAX];
    orc_levels(D0, n, kappa_b, s, sigma0, lvl, rml);
    long cnt[ORC_KMAX] = {0};
    for (long i = 0; i < n; ++i) cnt[lvl[i]]++;
    double V = box_volume(d, L);
    for (long i = 0; i < n; ++i) {
        int k = lvl[i];
        long c[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) c[a] = cell_of(x[d * i + a], L[a], orc_grid_n(L[a], cnt[k], V, occ));
        key[i] = pack_key(k, c[2], c[1], c[0]);
    }
    free(lvl);
}

/* ---- pair buffer ---- */
typedef struct { long row; int col; } orc_pair;
typedef struct { orc_pair* p; long n, cap; } pairbuf;

static void pb_push(pairbuf* b, long row, int col)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 1024;
        b->p = (orc_pair*)realloc(b->p, sizeof(orc_pair) * (size_t)b->cap);
    }
    b->p[b->n].row = row;
    b->p[b->n].col = col;
    b->n++;
}

static int pair_cmp(const void* a, const void* b)
{
    const orc_pair* x = (const orc_pair*)a;
    const orc_pair* y = (const orc_pair*)b;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    return 0;
}

static long pairs_to_csr(pairbuf* b, long n, long* rowptr, int* col, long cap)
{
    qsort(b->p, (size_t)b->n, sizeof(orc_pair), pair_cmp);
    if (b->n <= cap) {
        long t = 0;
        for (long i = 0; i <= n; ++i) {
            while (t < b->n && b->p[t].row < i) ++t;
            rowptr[i] = t;
        }
        for (long t2 = 0; t2 < b->n; ++t2) col[t2] = b->p[t2].col;
    }
    return b->n;
}

/* The listed set by definition: every ordered pair (i, j), i != j, whose
 * minimum-image distance is below rho_i + rho_j.  O(N^2).  Rows in ascending
 * i, columns in ascending j.  Returns the number of entries; writes them only
 * if it fits in cap. */
long orc_list_brute(const double* x, const double* D0, long n, int d, const double* L,
                    double kappa_b, double s, double sigma0,
                    long* rowptr, int* col, long cap)
{
    long t = 0;
    for (long i = 0; i < n; ++i) {
        if (t <= cap) rowptr[i] = t;
        double ri = orc_rho(D0[i], kappa_b, s, sigma0);
        for (long j = 0; j < n; ++j) {
            if (j == i) continue;
            double rj = orc_rho(D0[j], kappa_b, s, sigma0);
            if (orc_listed(&x[d * i], &x[d * j], d, L, ri, rj)) {
                if (t < cap) col[t] = (int)j;
                ++t;
            }
        }
    }
    if (t <= cap) rowptr[n] = t;
    return t;
}

/* One row of the listed set, by brute force over all j (O(N)). */
long orc_row_brute(const double* x, const double* D0, long n, int d, const double* L,
                   double kappa_b, double s, double sigma0, long i, int* col, long cap)
{
    long t = 0;
    double ri = orc_rho(D0[i], kappa_b, s, sigma0);
    for (long j = 0; j < n; ++j) {
        if (j == i) continue;
        double rj = orc_rho(D0[j], kappa_b, s, sigma0);
        if (orc_listed(&x[d * i], &x[d * j], d, L, ri, rj)) {
            if (t < cap) col[t] = (int)j;
            ++t;
        }
    }
    return t;
}

typedef struct { uint64_t key; long idx; } keyidx;
static int keyidx_cmp(const void* a, const void* b)
{
    const keyidx* x = (const keyidx*)a;
    const keyidx* y = (const keyidx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static long first_ge(const keyidx* a, long n, uint64_t key)
{
    long lo = 0, hi = n;
    while (lo < hi) {
        long mid = lo + (hi - lo) / 2;
        if (a[mid].key < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* The same listed set, found through the size classes: particle i scans, at
 * its own class and at every coarser class k, the cells within rho_i +
 * rho_max(k) (plus a margin far above rounding) of its position; the exact
 * predicate then decides.  A pair within one class is found from both ends; a
 * pair across classes only from the finer end, which records both
 * directions.  The result equals orc_list_brute (tested). */
long orc_list_grid(const double* x, const double* D0, long n, int d, const double* L,
                   double kappa_b, double s, double sigma0,
                   long* rowptr, int* col, long cap)
{
    return orc_list_grid_occ(x, D0, n, d, L, kappa_b, s, sigma0, 1.0, rowptr, col, cap);
}

long orc_list_grid_occ(const double* x, const double* D0, long n, int d, const double* L,
                       double kappa_b, double s, double sigma0, double occ,
                       long* rowptr, int* col, long cap)
{
    int* lvl = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double rml[ORC_KMAX];
    int nlev = orc_levels(D0, n, kappa_b, s, sigma0, lvl, rml);
    long cnt[ORC_KMAX] = {0};
    for (long i = 0; i < n; ++i) cnt[lvl[i]]++;
    double V = box_volume(d, L);
    long ng[ORC_KMAX][3];
    for (int k = 0; k < nlev; ++k)
        for (int a = 0; a < 3; ++a) ng[k][a] = a < d ? orc_grid_n(L[a], cnt[k], V, occ) : 1;
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) {
        long c[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) c[a] = cell_of(x[d * i + a], L[a], ng[lvl[i]][a]);
        ki[i].key = pack_key(lvl[i], c[2], c[1], c[0]);
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), keyidx_cmp);
    double Lmax = L[0];
    for (int a = 1; a < d; ++a) if (L[a] > Lmax) Lmax = L[a];

    pairbuf pb = {0, 0, 0};
    for (long i = 0; i < n; ++i) {
        double ri = orc_rho(D0[i], kappa_b, s, sigma0);
        for (int k = 0; k <= lvl[i]; ++k) {
            if (!(rml[k] > 0.0)) continue;
            double R = (ri + rml[k]) + 1e-9 * Lmax;
            long lo[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
            for (int a = 0; a < d; ++a) {
                long nn = ng[k][a];
                long l = (long)floor(((x[d * i + a] - R) / L[a]) * (double)nn);
                long h = (long)floor(((x[d * i + a] + R) / L[a]) * (double)nn);
                if (walled(a)) {   /* no wrap: clamp the window; edge cells hold what lies beyond */
                    if (l < 0) l = 0;
                    if (l > nn - 1) l = nn - 1;
                    if (h < 0) h = 0;
                    if (h > nn - 1) h = nn - 1;
                    lo[a] = l; cnt[a] = h - l + 1;
                } else if (h - l + 1 >= nn) { lo[a] = 0; cnt[a] = nn; }
                else { lo[a] = l; cnt[a] = h - l + 1; }
            }
            for (long cz = 0; cz < cnt[2]; ++cz)
                for (long cy = 0; cy < cnt[1]; ++cy)
                    for (long cx = 0; cx < cnt[0]; ++cx) {
                        long c0 = ((lo[0] + cx) % ng[k][0] + ng[k][0]) % ng[k][0];
                        long c1 = ((lo[1] + cy) % ng[k][1] + ng[k][1]) % ng[k][1];
                        long c2 = ((lo[2] + cz) % ng[k][2] + ng[k][2]) % ng[k][2];
                        uint64_t key = pack_key(k, c2, c1, c0);
                        for (long t = first_ge(ki, n, key); t < n && ki[t].key == key; ++t) {
                            long j = ki[t].idx;
                            if (j == i) continue;
                            double rj = orc_rho(D0[j], kappa_b, s, sigma0);
                            if (!orc_listed(&x[d * i], &x[d * j], d, L, ri, rj)) continue;
                            pb_push(&pb, i, (int)j);
                            if (k < lvl[i]) pb_push(&pb, j, (int)i);
                        }
                    }
        }
    }
    long P = pairs_to_csr(&pb, n, rowptr, col, cap);
    free(pb.p);
    free(ki);
    free(lvl);
    return P;
}

/* ------------------------------------------------------------------------ */
/* One pair of Eq. energy.  delta = 1 - r/d with d = kappa (D_i^0 + D_j^0)/2
 * when both spheres are mobile; with a frozen one, d is the mean of the two
 * contact diameters (size_at).  Returns delta; fills the minimum-image
 * displacement and r. */
static double pair_delta(const double* xi, const double* xj, double D0i, double D0j,
                         int d, const double* L, double kappa, double* dx, double* r, double* dd)
{
    double r2 = min_image(xi, xj, d, L, dx);
    *r = sqrt(r2);
    if (D0i > 0.0 && D0j > 0.0) *dd = kappa * (0.5 * (D0i + D0j));
    else *dd = 0.5 * (size_at(D0i, kappa) + size_at(D0j, kappa));
    return 1.0 - *r / *dd;
}

/* Row i's share of the sums, given its partners in ascending j.  gradient
 * d E / d x_i = - sum_j eps delta_ij / (d_ij r_ij) (x_i - x_j)_mi; energy and
 * kappa-derivative take j > i only:
 *   e_i = sum eps/2 delta^2,  k_i = sum eps delta (1 - delta) / kappa,
 * the latter from d delta / d kappa = (1 - delta)/kappa.  With a frozen
 * sphere in the pair, d d/d kappa = (mobile parts of D^0)/2 instead of d/kappa:
 *   k_i += eps delta (1 - delta) (mobile D_i^0 + mobile D_j^0)/2 / d,
 * and a frozen row takes no gradient (its coordinates are not variables). */
typedef struct { double g[3], e, k, md; } rowacc;

static void row_begin(rowacc* a) { a->g[0] = a->g[1] = a->g[2] = 0.0; a->e = a->k = a->md = 0.0; }

static void row_add(rowacc* a, long i, long j, const double* x, const double* D0, int d,
                    const double* L, double kappa, double eps)
{
    double dx[3], r, dd;
    double delta = pair_delta(&x[d * i], &x[d * j], D0[i], D0[j], d, L, kappa, dx, &r, &dd);
    if (!(delta > 0.0)) return;
    if (r > 0.0 && D0[i] > 0.0) {
        double coef = (eps * delta) / (dd * r);
        for (int c = 0; c < d; ++c) a->g[c] = a->g[c] - coef * dx[c];
    }
    if (j > i) {
        a->e = a->e + (0.5 * eps) * (delta * delta);
        if (D0[i] > 0.0 && D0[j] > 0.0)
            a->k = a->k + ((eps * delta) * (1.0 - delta)) / kappa;
        else
            a->k = a->k + (((eps * delta) * (1.0 - delta)) * (0.5 * (mobile_part(D0[i]) + mobile_part(D0[j])))) / dd;
    }
    if (delta > a->md) a->md = delta;
}

/* Row i's wall terms, after its pairs: for every axis a of the flat-wall
 * mask, the wall at 0 (h = x_a) then the wall at L_a (h = L_a - x_a); then the
 * curved container, h = R - |x - c| over its axes.  rad = kappa D^0/2 (F/2
 * frozen), delta = 1 - h/rad; when delta > 0:
 *   d E / d x_a = eps delta / rad * (- d h / d x_a)   (mobile rows: -+1 for the
 *   flat walls, (x_a - c_a)/|x - c| for the container, nothing at its centre),
 *   e_i += eps/2 delta^2,  k_i += eps delta (1 - delta)/kappa (mobile),
 * the latter from d delta / d kappa = (h/rad)/kappa. */
static void row_walls(rowacc* acc, long i, const double* x, const double* D0, int d, const double* L, double kappa,
                      double eps)
{
    if (!g_walls && !g_container) return;
    double rad = D0[i] > 0.0 ? kappa * (0.5 * D0[i]) : 0.5 * (-D0[i]);
    for (int a = 0; a < d; ++a) {
        if (!flat_wall(a)) continue;
        for (int side = 0; side < 2; ++side) {
            double h = side == 0 ? x[d * i + a] : L[a] - x[d * i + a];
            double delta = 1.0 - h / rad;
            if (!(delta > 0.0)) continue;
            if (D0[i] > 0.0) {
                double f = (eps * delta) / rad;
                acc->g[a] = side == 0 ? acc->g[a] - f : acc->g[a] + f;
                acc->k = acc->k + ((eps * delta) * (1.0 - delta)) / kappa;
            }
            acc->e = acc->e + (0.5 * eps) * (delta * delta);
            if (delta > acc->md) acc->md = delta;
        }
    }
    if (g_container) {
        /* curved wall: h = R - |x - c|; d h / d x_a = -(x_a - c_a)/|x - c| */
        double off[3];
        double rc = container_dist(&x[d * i], d, L, off);
        double h = container_R(d, L) - rc;
        double delta = 1.0 - h / rad;
        if (delta > 0.0) {
            if (D0[i] > 0.0) {
                if (rc > 0.0) {
                    double f = ((eps * delta) / rad) / rc;
                    for (int a = 0; a < d; ++a)
                        if (in_container(a, d)) acc->g[a] = acc->g[a] + f * off[a];
                }
                acc->k = acc->k + ((eps * delta) * (1.0 - delta)) / kappa;
            }
            acc->e = acc->e + (0.5 * eps) * (delta * delta);
            if (delta > acc->md) acc->md = delta;
        }
    }
}

static void finish_sums(const double* e, const double* k, const double* D0, long n,
                        double kappa, double mu, double* E, double* dEdk)
{
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) t[i] = mobile_part(D0[i]);
    double SD = orc_tree_sum(t, n);
    free(t);
    double Se = orc_tree_sum(e, n);
    double Sk = orc_tree_sum(k, n);
    if (E) *E = Se - mu * (kappa * SD);
    if (dEdk) *dEdk = Sk - mu * SD;
}

/* Eq. energy and its gradient by definition: all pairs, O(N^2). */
void orc_energy_grad_brute(const double* x, const double* D0, long n, int d, const double* L,
                           double kappa, double mu, double eps,
                           double* E, double* g, double* dEdk, double* maxdelta)
{
    double* e = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* k = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double md = 0.0;
    for (long i = 0; i < n; ++i) {
        rowacc a;
        row_begin(&a);
        for (long j = 0; j < n; ++j) if (j != i) row_add(&a, i, j, x, D0, d, L, kappa, eps);
        row_walls(&a, i, x, D0, d, L, kappa, eps);
        if (g) for (int c = 0; c < d; ++c) g[d * i + c] = a.g[c];
        e[i] = a.e;
        k[i] = a.k;
        if (a.md > md) md = a.md;
    }
    finish_sums(e, k, D0, n, kappa, mu, E, dEdk);
    if (maxdelta) *maxdelta = md;
    free(e);
    free(k);
}

/* The same sums over a listed superset of the overlapping pairs (CSR with
 * ascending columns): bit-identical to the brute-force version. */
void orc_energy_grad_list(const double* x, const double* D0, long n, int d, const double* L,
                          double kappa, double mu, double eps,
                          const long* rowptr, const int* col,
                          double* E, double* g, double* dEdk, double* maxdelta)
{
    double* e = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* k = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double md = 0.0;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 4096) reduction(max : md)
    for (long i = 0; i < n; ++i) {
        rowacc a;
        row_begin(&a);
        for (long t = rowptr[i]; t < rowptr[i + 1]; ++t) row_add(&a, i, col[t], x, D0, d, L, kappa, eps);
        row_walls(&a, i, x, D0, d, L, kappa, eps);
        if (g) for (int c = 0; c < d; ++c) g[d * i + c] = a.g[c];
        e[i] = a.e;
        k[i] = a.k;
        if (a.md > md) md = a.md;
    }
    finish_sums(e, k, D0, n, kappa, mu, E, dEdk);
    if (maxdelta) *maxdelta = md;
    free(e);
    free(k);
}

/* Row i alone, brute force over all j (for sampled checks at large N). */
void orc_row_grad(const double* x, const double* D0, long n, int d, const double* L,
                  double kappa, double eps, long i, double* g_i, double* e_i,
                  double* k_i, double* maxd_i)
{
    rowacc a;
    row_begin(&a);
    for (long j = 0; j < n; ++j) if (j != i) row_add(&a, i, j, x, D0, d, L, kappa, eps);
    row_walls(&a, i, x, D0, d, L, kappa, eps);
    for (int c = 0; c < d; ++c) g_i[c] = a.g[c];
    *e_i = a.e;
    *k_i = a.k;
    *maxd_i = a.md;
}

/* ------------------------------------------------------------------------ */
/* Adam (Kingma & Ba 2015, Algorithm 1) on n coordinates, with the running
 * products b1 = beta1^t and b2 = beta2^t already advanced to this step:
 *   m <- beta1 m + (1 - beta1) g;   v <- beta2 v + (1 - beta2) g^2
 *   p <- p - eta (m / (1 - b1)) / (sqrt(v / (1 - b2)) + adam_eps). */
void orc_adam_update(double* p, double* m, double* v, const double* g, long n,
                     double eta, double beta1, double beta2, double adam_eps,
                     double b1, double b2)
{
    double c1 = 1.0 - beta1, c2 = 1.0 - beta2;
    double h1 = 1.0 - b1, h2 = 1.0 - b2;
    for (long i = 0; i < n; ++i) {
        double gi = g[i];
        m[i] = beta1 * m[i] + c1 * gi;
        v[i] = beta2 * v[i] + c2 * (gi * gi);
        double mh = m[i] / h1;
        double vh = v[i] / h2;
        p[i] = p[i] - (eta * mh) / (sqrt(vh) + adam_eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Shrink to contact (Sec. II, App. A): with positions and D^0 fixed, the
 * largest kappa' <= kappa at which no pair overlaps is the smaller of kappa
 * and min_{i<j} r_ij / d_ij^0 (a pair touching exactly does not overlap).
 * Reading: that quotient is rounded, so the result is lowered by the factor
 * (1 - 2^-50) -- a few units in the last place -- which guarantees that a
 * binary64 re-evaluation at kappa_c finds no overlap at all.
 * A pair with one frozen sphere (fixed diameter F) touches at
 * kappa = (r - F/2) / (D_a^0 / 2); the subtraction can cancel bits, so that
 * quotient is lowered by (1 - 2^-40) first, and clamped at 0.  Two frozen
 * spheres do not depend on kappa and set no bound.  A mobile sphere at
 * distance h from a wall touches it at kappa = 2h / D^0 (clamped at 0). */
double orc_shrink_kappa(const double* x, const double* D0, long n, int d, const double* L,
                        double kappa, const long* rowptr, const int* col)
{
    double kc = kappa;
    for (long i = 0; i < n; ++i)
        for (long t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            long j = col[t];
            if (j <= i) continue;
            double dx[3];
            double r = sqrt(min_image(&x[d * i], &x[d * j], d, L, dx));
            double q;
            if (D0[i] > 0.0 && D0[j] > 0.0) {
                q = r / (0.5 * (D0[i] + D0[j]));
            } else if (D0[i] > 0.0 || D0[j] > 0.0) {
                double Da = D0[i] > 0.0 ? D0[i] : D0[j];
                double F = D0[i] > 0.0 ? -D0[j] : -D0[i];
                q = ((r - 0.5 * F) / (0.5 * Da)) * (1.0 - 0x1.0p-40);
                if (q < 0.0) q = 0.0;
            } else {
                continue;
            }
            if (q < kc) kc = q;
        }
    if (g_walls || g_container)
        for (long i = 0; i < n; ++i) {
            if (!(D0[i] > 0.0)) continue;
            if (g_container) {
                double off[3];
                double h = container_R(d, L) - container_dist(&x[d * i], d, L, off);
                double q = (2.0 * h) / D0[i];
                if (q < 0.0) q = 0.0;
                if (q < kc) kc = q;
            }
            for (int a = 0; a < d; ++a) {
                if (!flat_wall(a)) continue;
                for (int side = 0; side < 2; ++side) {
                    double h = side == 0 ? x[d * i + a] : L[a] - x[d * i + a];
                    double q = (2.0 * h) / D0[i];
                    if (q < 0.0) q = 0.0;
                    if (q < kc) kc = q;
                }
            }
        }
    return kc * (1.0 - 0x1.0p-50);
}

/* Solid-volume fraction of spheres (disks for d = 2) of diameters kappa D^0;
 * frozen spheres add their fixed volumes:
 *   phi = ((pi/6) kappa^3 sum_mobile D^3 + (pi/6) sum_frozen F^3) / V. */
double orc_phi(const double* D0, long n, int d, const double* L, double kappa)
{
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* f = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double V = solid_volume(d, L), phi;
    if (d == 2) {
        for (long i = 0; i < n; ++i) {
            double D = mobile_part(D0[i]), F = mobile_part(-D0[i]);
            t[i] = D * D;
            f[i] = F * F;
        }
        phi = ((((ORC_PI / 4.0) * (kappa * kappa)) * orc_tree_sum(t, n)) + (ORC_PI / 4.0) * orc_tree_sum(f, n)) / V;
    } else {
        for (long i = 0; i < n; ++i) {
            double D = mobile_part(D0[i]), F = mobile_part(-D0[i]);
            t[i] = (D * D) * D;
            f[i] = (F * F) * F;
        }
        phi = ((((ORC_PI / 6.0) * ((kappa * kappa) * kappa)) * orc_tree_sum(t, n)) + (ORC_PI / 6.0) * orc_tree_sum(f, n)) /
              V;
    }
    free(t);
    free(f);
    return phi;
}

/* ------------------------------------------------------------------------ */
void orc_params_default(orc_params* p)
{
    memset(p, 0, sizeof(*p));
    p->d = 3;
    p->L[0] = p->L[1] = p->L[2] = 1.0;
    p->phi0 = 0.05;
    p->eps = 1.0;
    p->beta1 = 0.9;
    p->beta2 = 0.999;
    p->adam_eps = 1e-8;
    p->skin_s = 0.1;
    p->skin_theta = 1.0;
    p->skin_abs = 20.0;
    p->lr_x = 1e-3;
    p->lr_kappa = 1e-3;
    p->delta_star0 = 1e-2;
    p->tol = 5e-4;
    p->Y = 2;
    p->X = 9;
    p->n_min = 2000;
    p->n_down = 3;
    p->n_cycles = 2;
    p->max_iters = 2000000;
}

/* Rebuild test (the list criterion above): a pair listed at kappa_b with
 * margin sigma_i + sigma_j stays non-overlapping while every sphere keeps
 * |x_i - x_i^b| + (kappa - kappa_b) D_i^0 / 2 <= theta sigma_i, theta <= 1.
 * Returns 1 if some sphere broke it (1e-9 margins cover rounding).  A frozen
 * sphere neither moves nor grows and never breaks it. */
static int skin_spent(const double* x, const double* xb, const double* D0, long n, int d, const double* L,
                      double kappa, double kb, double s, double th, double sigma0)
{
    for (long i = 0; i < n; ++i) {
        if (!(D0[i] > 0.0)) continue;
        double dx[3];
        double disp = sqrt(min_image(&x[d * i], &xb[d * i], d, L, dx)) * (1.0 + 1e-9);
        double sig = th * (s * kb * D0[i] + sigma0) * (1.0 - 1e-9);
        if (disp + (kappa - kb) * D0[i] * 0.5 * (1.0 + 1e-9) > sig) return 1;
    }
    return 0;
}

/* Rung table (reading of App. A: a short descent of mu in discrete rungs,
 * then mu cycles, then a final relaxation at mu = 0 with a smaller learning
 * rate that runs until the stopping criterion).  Rung 0 lasts n_trig of
 * Eq. trigger (at least n_min); every later rung n_trig/4 (at least n_min).
 * The target overlap falls tenfold per rung, the learning rate halves. */
typedef struct { double dstar, lrs; long budget; int final; } rung;

static int build_rungs(const orc_params* p, long n, rung* R, int cap)
{
    double nt = orc_n_trig(n, p->d, p->Y, p->X);
    long b0 = (long)ceil(nt);
    if (b0 < p->n_min) b0 = p->n_min;
    long bq = (long)ceil(nt / 4.0);
    if (bq < p->n_min) bq = p->n_min;
    int c = 0;
    double ds = p->delta_star0, lrs = 1.0;
    R[c].dstar = ds; R[c].lrs = lrs; R[c].budget = b0; R[c].final = 0; ++c;
    for (int r = 1; r <= p->n_down && c < cap; ++r) {
        ds = ds / 10.0;
        lrs = lrs * 0.5;
        R[c].dstar = ds; R[c].lrs = lrs; R[c].budget = bq; R[c].final = 0; ++c;
    }
    for (int cy = 0; cy < p->n_cycles && c + 2 < cap; ++cy) {
        R[c].dstar = ds * 10.0; R[c].lrs = lrs; R[c].budget = bq; R[c].final = 0; ++c;
        R[c].dstar = ds; R[c].lrs = lrs; R[c].budget = bq; R[c].final = 0; ++c;
    }
    R[c].dstar = 0.0; R[c].lrs = lrs * 0.5; R[c].budget = p->max_iters; R[c].final = 1; ++c;
    return c;
}

/* Adam on the coordinates of the mobile spheres; frozen ones keep their
 * positions and moments. */
static void adam_positions(double* x, double* m, double* v, const double* g, const double* D0, long n, int d,
                           double eta, const orc_params* p, double b1, double b2)
{
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long i = 0; i < n; ++i)
        if (D0[i] > 0.0)
            orc_adam_update(&x[d * i], &m[d * i], &v[d * i], &g[d * i], d, eta, p->beta1, p->beta2, p->adam_eps, b1,
                            b2);
}

static long build_list(const double* x, const double* D0, long n, int d, const double* L,
                       double kb, double s, double sigma0, long** rowptr, int** col, long* cap)
{
    for (;;) {
        long P = orc_list_grid(x, D0, n, d, L, kb, s, sigma0, *rowptr, *col, *cap);
        if (P <= *cap) return P;
        *cap = P + P / 2 + 16;
        *col = (int*)realloc(*col, sizeof(int) * (size_t)(*cap));
    }
}

/* The whole protocol.  trace (optional): per iteration {E, max delta, kappa,
 * dE/dkappa}.  x_io: initial positions if x_given, and the positions at stop
 * on return.  Returns 0 on success, 1 on bad input, 2 if the periodic-image
 * rule is broken (the largest interaction diameter must stay below half the
 * box edge, Sec. II). */
int orc_run(const orc_params* p, const double* D0, long n, uint64_t seed,
            double* x_io, int x_given, orc_result* res, double* trace, long trace_cap)
{
    int d = p->d;
    const double* L = p->L;
    if (n < 1 || (d != 2 && d != 3)) return 1;
    int walls_before = g_walls, container_before = g_container;
    g_walls = p->walls;
    g_container = p->container;
    long nd = n * d;
    double* x = (double*)malloc(sizeof(double) * (size_t)nd);
    double* m = (double*)calloc((size_t)nd, sizeof(double));
    double* v = (double*)calloc((size_t)nd, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * (size_t)nd);
    double* xb = (double*)malloc(sizeof(double) * (size_t)nd);
    long cap = 64 * n + 1024;
    long* rowptr = (long*)malloc(sizeof(long) * (size_t)(n + 1));
    int* col = (int*)malloc(sizeof(int) * (size_t)cap);
    if (x_given) memcpy(x, x_io, sizeof(double) * (size_t)nd);
    else orc_init_positions(seed, n, d, L, x);

    double mom[3];
    orc_moments(D0, n, mom);
    double SD = mom[0], SD3 = mom[1], SD4 = mom[2];
    double Dref = SD4 / SD3;
    double Neff = SD3 / ((Dref * Dref) * Dref);
    double kappa = orc_kappa0(D0, n, d, L, p->phi0);
    double sigma0 = p->skin_abs * ((p->lr_x * kappa) * Dref);
    if (p->kappa_init > 0.0) kappa = p->kappa_init;   /* sigma0 stays that of kappa_0 */
    double mk = 0.0, vk = 0.0, b1 = 1.0, b2 = 1.0;
    double s = p->skin_s, th = p->skin_theta;
    double Lmin = INFINITY;   /* the periodic-image rule concerns periodic axes only */
    for (int a = 0; a < d; ++a) if (!walled(a) && L[a] < Lmin) Lmin = L[a];

    long n_mobile = 0;
    for (long i = 0; i < n; ++i) n_mobile += D0[i] > 0.0;
    rung R[64];
    int nr = build_rungs(p, n_mobile, R, 60);
    long it = 0, rebuilds = 0;
    int need = 1, stopped = 0, status = 0;
    double kb = kappa, E = 0.0, md = 0.0, dEdk = 0.0;
    for (int r = 0; r < nr && !stopped && it < p->max_iters; ++r) {
        double kr = kappa;
        double mu = R[r].dstar > 0.0 ? (((3.0 * R[r].dstar) * p->eps) * Neff) / (kr * SD) : 0.0;
        double eta_x = ((p->lr_x * R[r].lrs) * kr) * Dref;
        double eta_k = (p->lr_kappa * R[r].lrs) * kr;
        for (long t = 0; t < R[r].budget && it < p->max_iters; ++t) {
            if (need) {
                double rmax = orc_rho(D0[0], kappa, s, sigma0);
                for (long i = 1; i < n; ++i) {
                    double q = orc_rho(D0[i], kappa, s, sigma0);
                    if (q > rmax) rmax = q;
                }
                if (!(4.0 * rmax < Lmin)) { status = 2; goto done; }
                build_list(x, D0, n, d, L, kappa, s, sigma0, &rowptr, &col, &cap);
                memcpy(xb, x, sizeof(double) * (size_t)nd);
                kb = kappa;
                ++rebuilds;
                need = 0;
            }
            orc_energy_grad_list(x, D0, n, d, L, kappa, mu, p->eps, rowptr, col, &E, g, &dEdk, &md);
            if (trace && it < trace_cap) {
                trace[4 * it + 0] = E;
                trace[4 * it + 1] = md;
                trace[4 * it + 2] = kappa;
                trace[4 * it + 3] = dEdk;
            }
            if (R[r].final && md < p->tol) { stopped = 1; break; }
            b1 = b1 * p->beta1;
            b2 = b2 * p->beta2;
            adam_positions(x, m, v, g, D0, n, d, eta_x, p, b1, b2);
            for (long i = 0; i < n; ++i)
                for (int a = 0; a < d; ++a)
                    if (!walled(a)) x[d * i + a] = orc_wrap(x[d * i + a], L[a]);
            orc_adam_update(&kappa, &mk, &vk, &dEdk, 1, eta_k, p->beta1, p->beta2, p->adam_eps, b1, b2);
            ++it;
            need = need || skin_spent(x, xb, D0, n, d, L, kappa, kb, s, th, sigma0);
        }
    }
    {
        /* shrink to contact with a fresh list at the final state */
        build_list(x, D0, n, d, L, kappa, s, sigma0, &rowptr, &col, &cap);
        double kc = orc_shrink_kappa(x, D0, n, d, L, kappa, rowptr, col);
        res->iters = it;
        res->rebuilds = rebuilds;
        res->stopped = stopped;
        res->kappa = kappa;
        res->max_delta = md;
        res->energy = E;
        res->kappa_c = kc;
        res->phi = orc_phi(D0, n, d, L, kc);
        memcpy(x_io, x, sizeof(double) * (size_t)nd);
    }
done:
    g_walls = walls_before;
    g_container = container_before;
    free(x); free(m); free(v); free(g); free(xb); free(rowptr); free(col);
    return status;
}

/* A bounded sample of the protocol for timing the CPU baseline: `iters`
 * iterations of the loop body of orc_run (list build when the skin budget is
 * spent, Eq. energy and gradient, Adam on x and kappa) from positions x at
 * kappa, with fixed rung values mu, eta_x, eta_kappa and zero Adam moments.
 * Returns the number of list builds, or -1 if the periodic-image rule fails. */
long orc_sample_iterations(const orc_params* p, const double* D0, long n, double* x, double kappa,
                           double mu, double eta_x, double eta_k, double sigma0, long iters)
{
    int d = p->d;
    const double* L = p->L;
    long nd = n * d;
    double* m = (double*)calloc((size_t)nd, sizeof(double));
    double* v = (double*)calloc((size_t)nd, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * (size_t)nd);
    double* xb = (double*)malloc(sizeof(double) * (size_t)nd);
    long cap = 64 * n + 1024;
    long* rowptr = (long*)malloc(sizeof(long) * (size_t)(n + 1));
    int* col = (int*)malloc(sizeof(int) * (size_t)cap);
    double mk = 0.0, vk = 0.0, b1 = 1.0, b2 = 1.0, kb = kappa, E, dEdk, md;
    double s = p->skin_s, th = p->skin_theta;
    double Lmin = L[0];
    for (int a = 1; a < d; ++a) if (L[a] < Lmin) Lmin = L[a];
    long builds = 0;
    int need = 1;
    for (long t = 0; t < iters; ++t) {
        if (need) {
            double rmax = 0.0;
            for (long i = 0; i < n; ++i) {
                double q = orc_rho(D0[i], kappa, s, sigma0);
                if (q > rmax) rmax = q;
            }
            if (!(4.0 * rmax < Lmin)) { builds = -1; break; }
            build_list(x, D0, n, d, L, kappa, s, sigma0, &rowptr, &col, &cap);
            memcpy(xb, x, sizeof(double) * (size_t)nd);
            kb = kappa;
            ++builds;
            need = 0;
        }
        orc_energy_grad_list(x, D0, n, d, L, kappa, mu, p->eps, rowptr, col, &E, g, &dEdk, &md);
        b1 = b1 * p->beta1;
        b2 = b2 * p->beta2;
        adam_positions(x, m, v, g, D0, n, d, eta_x, p, b1, b2);
        for (long i = 0; i < n; ++i)
            for (int a = 0; a < d; ++a)
                if (!walled(a)) x[d * i + a] = orc_wrap(x[d * i + a], L[a]);
        orc_adam_update(&kappa, &mk, &vk, &dEdk, 1, eta_k, p->beta1, p->beta2, p->adam_eps, b1, b2);
        need = need || skin_spent(x, xb, D0, n, d, L, kappa, kb, s, th, sigma0);
    }
    free(m); free(v); free(g); free(xb); free(rowptr); free(col);
    return builds;
}
