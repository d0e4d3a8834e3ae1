/*
 * rcp.h -- C ABI of the B300 (sm_103a) implementation of the Adam-based
 * Clarke-Wiley inflation protocol for random close packings of polydisperse
 * spheres (arxiv 2608.12235, Sec. II and Appendix A).
 *
 * One handle holds one packing: N spheres of fixed relative diameters D_i^0
 * in a periodic box, their positions x_i, the common diameter scale kappa
 * (D_i = kappa D_i^0), the Adam moments, and the neighbour structure.  All
 * device memory belongs to the handle; every pointer argument belongs to the
 * caller and is only read or written during the call (copied, never kept).
 *
 * Conventions for every entry point:
 *   - the return value is an rcp_status; RCP_OK on success.  On failure a
 *     message is kept in the handle (rcp_last_error) and no output is written
 *     unless stated;
 *   - positions are row-major [N][d] doubles in the caller's particle order;
 *   - work is issued on the handle's CUDA stream (rcp_set_stream); calls that
 *     return host data synchronise that stream before returning;
 *   - `on_device` = 1 means the pointer arguments of that call are device
 *     pointers on the handle's device (outputs are then written
 *     asynchronously on the handle's stream); 0 means host pointers;
 *   - d is 3 or 2 (disks; the paper's quantitative results are 3D, Sec. II
 *     shows disks among its domains); other d return RCP_ERR_UNSUPPORTED.
 *     Positions, gradients and moments then have two columns at the boundary.
 */
#ifndef RCP_H
#define RCP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rcp_ctx* rcp_handle;

typedef enum {
    RCP_OK = 0,
    RCP_ERR_ARG = 1,         /* an argument is invalid (message says which) */
    RCP_ERR_IMAGE = 2,       /* an interaction diameter reaches half a box edge: the
                                largest sphere would meet its own periodic image (Sec. II) */
    RCP_ERR_OOM = 3,         /* device allocation failed */
    RCP_ERR_NAN = 4,         /* a non-finite energy or gradient appeared */
    RCP_ERR_CAPACITY = 5,    /* a fixed-size internal table is too small */
    RCP_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    RCP_ERR_MAXITER = 7,     /* the iteration cap was reached before the stopping criterion */
    RCP_ERR_CUDA = 8,        /* a CUDA runtime call failed (message has its text) */
    RCP_ERR_UNSUPPORTED = 9  /* valid but not implemented here (e.g. d other than 2 or 3) */
} rcp_status;

typedef enum {
    RCP_FP64 = 0,   /* all arithmetic in binary64, canonical summation order:
                       bit-identical to the CPU oracle */
    RCP_MIXED = 1   /* pair geometry in binary32 on fixed-point cell-relative
                       offsets, Adam moments in binary32; positions, global
                       reductions and the stopping test in binary64 */
} rcp_precision;

/* Optimiser and schedule settings.  Appendix A names the ingredients (Adam on
 * the coordinates and kappa, mu annealed in rungs then cycled, a learning rate
 * reduced over the run, rung budgets from Eq. trigger with a minimum count,
 * the 5e-4 stop) but leaves the constants to its code; the defaults below are
 * this implementation's readings. */
typedef struct {
    int       precision;    /* rcp_precision */
    double    phi0;         /* initial packing fraction: sets kappa_0 (default 0.05) */
    double    eps;          /* overlap stiffness epsilon of Eq. energy (1) */
    double    beta1;        /* Adam first-moment decay (0.9) */
    double    beta2;        /* Adam second-moment decay (0.999) */
    double    adam_eps;     /* Adam denominator guard (1e-8) */
    double    skin_s;       /* size-proportional Verlet skin fraction s (0.1) */
    double    skin_theta;   /* rebuild when a sphere's displacement plus its share
                               (kappa - kappa_b) D_i/2 of the growth exceeds theta of
                               its skin sigma_i; theta <= 1 keeps every overlapping
                               pair listed (1) */
    double    skin_abs;     /* absolute skin sigma0 in units of the first rung's
                               position learning rate (20) */
    double    lr_x;         /* position learning rate in units of kappa D_ref,
                               D_ref = sum D^4 / sum D^3 (1e-3) */
    double    lr_kappa;     /* kappa learning rate in units of kappa (1e-3) */
    double    delta_star0;  /* target mean overlap of the first rung (1e-2) */
    double    tol;          /* stop when max fractional overlap < tol (5e-4, App. A) */
    int       Y, X;         /* Eq. trigger constants: (2, 9) default, (3, 24) long */
    long long n_min;        /* minimum rung budget (2000) */
    int       n_down;       /* rungs after the first, mu falling tenfold each (3) */
    int       n_cycles;     /* mu cycles after the descent (2) */
    long long max_iters;    /* cap on Adam steps (2000000) */
    int       chunk;        /* iterations per CUDA-graph replay (32) */
    double    cell_occupancy; /* spheres per cell each size class's grid aims at:
                                 cells are the smallest power-of-two grid with at
                                 least this many per cell on average (1) */
    int       placement;    /* initial positions: 0 uniform in the box (default);
                               1 without overlap at phi0 (App. A starts the run from
                               a dilute configuration with no overlaps): rounds of
                               random sequential addition, larger spheres first,
                               round 0 being the uniform draw */
    int       place_rounds; /* most placement rounds before rcp_create gives up
                               with RCP_ERR_CAPACITY (10000) */
    int       walls;        /* boundary (Sec. II: each axis periodic or bounded by a
                               hard wall): bit a set bounds axis a by flat walls at 0
                               and L_a -- no minimum image and no wrap there, and a
                               sphere closer than its contact radius rad = kappa
                               D^0/2 to a wall overlaps it by delta = 1 - h/rad (h
                               the distance to the wall), adding eps/2 delta^2 to
                               Eq. energy; shrink to contact also stops at the first
                               wall contact and placement keeps spheres off the
                               walls.  Positions on walled axes should stay within
                               one box edge of the box; in RCP_MIXED a bounded
                               axis's fixed-point record spans [-L_a/2, 3 L_a/2)
                               (a position outside saturates to its end) and the
                               wall terms are taken in two-term binary32.  Only
                               the bits of the d axes; either precision (0:
                               periodic box) */
    int       container;    /* curved hard wall (Sec. II, Fig. 2): 0 none; 1 a ball
                               over every axis (a disk when d = 2); 2 a cylinder
                               about the z axis (d = 3).  Radius R = min L_a/2 over
                               its axes, centre at the box centre; its axes take no
                               minimum image or wrap; a sphere with h = R - |x - c|
                               below its contact radius overlaps the wall by
                               delta = 1 - h/rad as for a flat wall; kappa_0 and
                               phi use the container's volume.  Start from
                               placement = 1 (a uniform draw over the box leaves
                               spheres outside).  Either precision, the container's
                               axes recorded in RCP_MIXED as walled axes are */
} rcp_config;

/* When rcp_run returns early. */
typedef struct {
    long long max_iters;    /* at most this many Adam steps in this call (0: no limit) */
    double    max_seconds;  /* wall-clock limit for this call (0: none) */
    int       shrink;       /* 1: shrink to contact once the stopping criterion fires */
} rcp_stop;

typedef struct {
    long long iters;        /* Adam steps taken since creation */
    long long rebuilds;     /* neighbour-structure builds since creation */
    long long pairs;        /* listed ordered pairs at the last build */
    int       stopped;      /* 1 once the stopping criterion of App. A has fired */
    double    kappa;        /* current kappa */
    double    max_delta;    /* max fractional overlap 1 - r/d at the last evaluation */
    double    energy;       /* Eq. energy at the last evaluation */
    double    kappa_c;      /* shrink-to-contact kappa (0 until computed) */
    double    phi;          /* shrink-to-contact packing fraction (0 until computed) */
    double    seconds;      /* wall time of this call */
    long long launches;     /* CUDA kernels launched by this call (each kernel of a
                               replayed graph counts once per replay) */
} rcp_result;

/* Optimiser scalars, for checkpoint and resume (rcp_state / rcp_load_state). */
typedef struct {
    long long t;            /* Adam steps taken */
    double    kappa, m_kappa, v_kappa;
    double    b1, b2;       /* running products beta1^t, beta2^t */
    int       rung;         /* index of the current rung of the schedule */
    long long rung_start;   /* value of t when the current rung began */
    double    kappa_rung;   /* kappa when the current rung began */
    int       stopped;      /* 1 once the stopping criterion has fired */
} rcp_scalars;

/* Fill *cfg with the defaults listed above. */
rcp_status rcp_config_default(rcp_config* cfg);

/* Create a packing (Sec. II: the caller supplies the N relative diameters,
 * the dimension and the boundary; here the boundary is a periodic box).
 *   diameters: host array of N positive finite relative diameters D_i^0;
 *   N >= 1; d is 3 (spheres) or 2 (disks; else RCP_ERR_UNSUPPORTED); every
 *   position, gradient and moment array of the other calls has d columns;
 *   box: host array of d positive box edges;
 *   seed: positions are uniform in the box, coordinate a of sphere i taken
 *         from output d i + a of SplitMix64 seeded with `seed`;
 *   cfg: NULL for the defaults;
 *   kappa_0 is set so that the packing fraction equals cfg->phi0.
 * On success *out receives the handle, which owns a new non-blocking stream
 * on the current device. */
rcp_status rcp_create(const double* diameters, long long N, int d, const double* box,
                      unsigned long long seed, const rcp_config* cfg, rcp_handle* out);

/* Free every resource of the handle.  NULL is accepted. */
rcp_status rcp_destroy(rcp_handle h);

/* Issue the handle's work on `stream` (a cudaStream_t of the handle's
 * device; NULL selects the handle's own stream; cudaStreamLegacy selects the
 * legacy default stream, on which graphs cannot be captured: rcp_run then
 * replays its graph on the handle's own stream, ordered before and after
 * with events).  Captured graphs are re-captured on the next call that needs
 * them. */
rcp_status rcp_set_stream(rcp_handle h, void* stream);

/* Replace the positions (N x 3, wrapped into the box) and optionally kappa
 * (kappa > 0; pass a value <= 0 to keep it).  The neighbour structure is
 * checked against the new state before the next evaluation. */
rcp_status rcp_set_positions(rcp_handle h, const double* x, double kappa, int on_device);

/* Build the size-stratified cell levels and the Verlet list at the current
 * state (App. A uses a k-d tree rebuilt on accumulated displacement; this is
 * the B300 replacement).  The list holds every ordered pair (i, j), i != j,
 * whose minimum-image distance is below rho_i + rho_j, rho_i = kappa D_i^0
 * (1/2 + s) + sigma0. */
rcp_status rcp_build_neighbors(rcp_handle h);

/* Evaluate Eq. energy at the current state with growth weight `mu`:
 *   E = eps/2 sum_{i<j} delta_ij^2 Theta(delta_ij) - mu kappa sum_i D_i^0,
 *   delta_ij = 1 - r_ij / d_ij, d_ij = kappa (D_i^0 + D_j^0)/2,
 * its gradient grad_x[N][3] = dE/dx_i, dE/dkappa, and the largest fractional
 * overlap max(0, max delta_ij).  Any output pointer may be NULL.  With
 * on_device = 1 all non-NULL outputs are device pointers. */
rcp_status rcp_energy_grad(rcp_handle h, double mu, double* E, double* grad_x,
                           double* dE_dkappa, double* max_delta, int on_device);

/* Evaluate at a state given on the device: positions x_dev [N][3] (inside
 * or outside the box; wrapped) and kappa_dev (one double) become the
 * handle's state, the neighbour structure is rebuilt if the skin test asks
 * for it, and E, grad_x[N][3], dE/dkappa and max delta are written to the
 * given device pointers (any of them may be NULL).  This is the forward of
 * the torch.autograd binding: one fused pass gives the energy and both
 * gradients.  Reads one flag back to the host (the rebuild decision). */
rcp_status rcp_energy_grad_at(rcp_handle h, const double* x_dev, const double* kappa_dev, double mu,
                              double* E, double* grad_x, double* dE_dkappa, double* max_delta);

/* One Adam step (Kingma & Ba, Algorithm 1) on every coordinate and on kappa
 * with the given gradient (grad_x[N][3], host or device per on_device) and
 * step sizes lr_x (length units) and lr_kappa; positions are wrapped into the
 * box.  Advances t and the bias-correction products. */
rcp_status rcp_adam_step(rcp_handle h, const double* grad_x, double dE_dkappa,
                         double lr_x, double lr_kappa, int on_device);

/* Run the protocol of App. A from the current state: the rung schedule, then
 * the final rung until the max fractional overlap is below cfg.tol, then (if
 * stop->shrink) shrink kappa to contact and compute phi.  Returns early when
 * a limit in *stop is reached (stop may be NULL: no limits, shrink on); a
 * later call resumes bit-exactly.  Returns RCP_ERR_MAXITER if cfg.max_iters
 * is reached first.  *out (may be NULL) receives the summary. */
rcp_status rcp_run(rcp_handle h, const rcp_stop* stop, rcp_result* out);

/* Instrumented run: like rcp_run with stop = {iters, 0, 0}, but every
 * iteration is launched on its own (no graph) with CUDA events around the
 * pair kernel.  *ms_pair receives the summed pair-kernel time, *ms_iter the
 * summed time of whole iterations (pair kernel, reductions, kappa step),
 * *launches the number of pair-kernel launches timed.  The iterations are
 * real: the state advances exactly as under rcp_run. */
rcp_status rcp_profile(rcp_handle h, long long iters, double* ms_pair, double* ms_iter,
                       long long* launches);

/* Shrink to contact at the current state (Sec. II, App. A): kappa_c is the
 * smaller of kappa and min_{i<j} r_ij / d_ij^0, lowered by the factor
 * (1 - 2^-50) so that a binary64 re-evaluation finds no overlap; phi is the
 * solid-volume fraction at kappa_c.  Positions and kappa are not changed. */
rcp_status rcp_shrink(rcp_handle h, double* kappa_c, double* phi);

/* Copy the state to host arrays (any pointer may be NULL): x and the Adam
 * moments m, v as [N][3] doubles (binary32 moments are widened), and the
 * optimiser scalars. */
rcp_status rcp_state(rcp_handle h, double* x, double* m, double* v, rcp_scalars* s);

/* Restore a state written by rcp_state (host arrays; NULL keeps a part). */
rcp_status rcp_load_state(rcp_handle h, const double* x, const double* m, const double* v,
                          const rcp_scalars* s);

/* Copy the current Verlet list to the host as CSR: rowptr[N+1] and col[P]
 * with ascending columns per row.  *P receives the entry count; col is
 * written only if P <= cap.  Builds the list first if none exists. */
rcp_status rcp_neighbors(rcp_handle h, long long* rowptr, int* col, long long cap,
                         long long* P);

/* Copy the per-sphere cell keys of the last build: size class in bits 57-61,
 * then the z, y, x cell indices of that class's grid in 19 bits each. */
rcp_status rcp_cell_keys(rcp_handle h, unsigned long long* keys);

/* Number of spheres. */
long long rcp_size(rcp_handle h);

/* Dimension d given at creation (2 or 3; 0 for NULL). */
int rcp_dim(rcp_handle h);

/* ---- the sequential multimodal cascade (Sec. IV) ----
 * The paper packs a multimodal grading class by class, coarsest first: the
 * finer class is seated into the voids of the packed coarser spheres and
 * inflated to contact with those held fixed, then everything is released and
 * relaxed together, and so on down the classes.  The calls below give the
 * "held fixed" part: frozen spheres keep their positions and a contact
 * diameter that kappa does not scale.  Both precisions: the mixed path
 * carries the frozen flag in the sign of the record's D^0 and runs a pair
 * kernel that tells the contact diameters apart whenever the packing holds
 * frozen spheres. */

/* Create a seated packing: Nf >= 1 frozen spheres (internal indices
 * 0..Nf-1) and N >= 1 mobile ones (indices Nf..Nf+N-1; every array of the
 * other calls has Nf + N rows in that order).
 *   fixed_d: host [Nf] contact diameters F_i > 0 of the frozen spheres;
 *   fixed_x: host [Nf][d] their positions (wrapped into the box);
 *   diameters: host [N] relative diameters D_i^0 of the mobile spheres;
 *   d, box, seed: as for rcp_create (the uniform draw covers all Nf + N
 *         indices; the frozen rows are then replaced by fixed_x);
 *   cfg: required, either precision, with or without walls or a container.
 * Pairs with a frozen sphere have d_ij = (F_i + kappa D_j^0)/2 (or (F_i +
 * F_j)/2), so dE/dkappa takes (mobile D^0)/2 from them; a frozen sphere's
 * gradient is zero and Adam does not move it; the growth term -mu kappa sum
 * D^0, the moments that scale the schedule (D_ref, N_eff), kappa_0 (phi0 of
 * the mobile spheres alone) and the rung budgets (Eq. trigger with the mobile
 * count) take the mobile spheres only; cfg->placement = 1 places the mobile
 * spheres around the frozen ones, which count as placed from the start.
 * Shrink to contact bounds kappa by every pair with a mobile sphere (a pair
 * with a frozen one touches at kappa = (r - F/2)/(D^0/2), lowered by
 * (1 - 2^-40)); phi adds the frozen spheres' fixed volumes. */
rcp_status rcp_create_seated(const double* fixed_d, const double* fixed_x, long long Nf, const double* diameters,
                             long long N, int d, const double* box, unsigned long long seed,
                             const rcp_config* cfg, rcp_handle* out);

/* Number of frozen spheres (0 for rcp_create handles and NULL). */
long long rcp_frozen(rcp_handle h);

/* The whole cascade.  cls[i] in 0..C-1 is the class of sphere i (class 0
 * first; every class non-empty).  Stage 0 packs class 0 alone (rcp_create,
 * seed).  Stage s >= 1 seats class s (rcp_create_seated with seed + s, the
 * packed spheres frozen in ascending caller index, then the class in
 * ascending caller index), runs it to the stop and shrinks it; then releases
 * every sphere: rcp_create of the contact diameters with phi0 = the seated
 * phi and placement off, positions from the seated run with kappa = 1, run to
 * the stop and shrunk.  After each stage the diameters are the contact
 * diameters kappa_c D.  cfg: required, either precision (every stage runs
 * in it).
 *   x_out: host [N][d] final positions, diam_out: host [N] final contact
 *   diameters (caller order); phi_out, iters_out (may be NULL): host [2C-1]
 *   phi and Adam steps of the stages in order: pack, seat 1, release 1,
 *   seat 2, release 2, ...
 * Returns RCP_ERR_MAXITER if a stage does not reach the stopping criterion. */
rcp_status rcp_cascade(const double* diameters, const int* cls, long long N, int d, const double* box,
                       unsigned long long seed, const rcp_config* cfg, double* x_out, double* diam_out,
                       double* phi_out, long long* iters_out);

/* ---- batches: many independent packings in one graph of batched kernels ---- */
typedef struct rcp_batch_ctx* rcp_batch;

/* Group B existing handles (same device, same precision; each at most ~8192
 * block partial sums, i.e. N up to ~2e6 in binary64 or ~2.5e5 in mixed
 * precision) for rcp_batch_run.  The handles keep their state and ownership;
 * destroy the batch before its handles.  autotune = 1 times, on the first
 * run, the long-row threshold of the mixed pair kernel (16, 32, 64, 128) and
 * the iterations per graph replay (8, 16, 32, 64) and keeps the fastest.
 * A failure message is left in rcp_last_error(hs[0]). */
rcp_status rcp_batch_create(rcp_handle* hs, int B, int autotune, rcp_batch* out);

/* Advance every packing of the batch as rcp_run would (its own rung schedule,
 * stopping test, rebuilds, and shrink to contact once it stops), all of them
 * in each replay of one CUDA graph whose per-iteration work is one batched
 * pair kernel and one batched kappa step.  A packing's trajectory is
 * bit-identical to running it alone with the same long-row threshold.
 * outs (may be NULL) receives B summaries; outs[0].launches counts the
 * batch's kernel launches.  Returns the first non-OK status of a packing. */
rcp_status rcp_batch_run(rcp_batch b, const rcp_stop* stop, rcp_result* outs);

/* The tuned long-row threshold and iterations per replay. */
rcp_status rcp_batch_tuning(rcp_batch b, int* long_row, int* chunk);

/* Free the batch (not its handles).  NULL is accepted. */
rcp_status rcp_batch_destroy(rcp_batch b);

/* Message of the last failure on this batch ("" if none). */
const char* rcp_batch_last_error(rcp_batch b);

/* Largest N accepted by rcp_energy_grad_noalloc. */
#define RCP_NOALLOC_MAX_N (1LL << 21)

/* Binary64 evaluation that allocates no memory (the paper has no counterpart:
 * this is a service for callers that cannot allocate device memory -- code
 * running inside a memory pool another runtime has fully reserved, hosts that
 * partition device memory once at start-up, or callers that must not enter
 * the allocator while another library holds it).  No handle is involved and
 * no cudaMalloc, cudaFree or allocating library routine is called.
 *
 * Computes, from caller-owned DEVICE buffers, what rcp_energy_grad computes
 * in RCP_FP64 mode for a periodic d = 3 box without walls, container or
 * frozen spheres (the only case it covers): Eq. energy E, grad_x[N][3] =
 * dE/dx_i, dE/dkappa and max(0, max delta_ij), bit for bit, over the CSR
 * list rowptr[N+1] / col[P] (unsigned 32-bit, ascending columns per row).
 * The list must be a full (symmetric) list holding every overlapping pair in
 * both rows -- j in row i and i in row j -- as rcp_neighbors' list does: a
 * row's energy share counts its partners j > i, its gradient all partners,
 * so a half list gives wrong gradients without an error.
 *   x: [N][3] positions inside the box; D0: [N] relative diameters;
 *   box: HOST array of 3 box edges; kappa > 0; mu and eps as in Eq. energy;
 *   E, dE_dkappa, max_delta: device pointers to one double each (may be NULL);
 *   stream: the cudaStream_t to run on (NULL: the legacy default stream).
 * Work is asynchronous on `stream`; outputs are valid once it completes.
 *
 * Scratch lives in a fixed static device array inside the library (about
 * 192 KiB, held by every GPU that loads the library until the process exits)
 * sized for N <= RCP_NOALLOC_MAX_N; larger N returns RCP_ERR_CAPACITY.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and caches it, so make that
 * first call before any stream capture.  Every call shares the one array: two
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads) race and both results are undefined; serialize them. */
rcp_status rcp_energy_grad_noalloc(const double* x, const double* D0, long long N, const double* box,
                                   double kappa, double mu, double eps, const unsigned int* rowptr,
                                   const unsigned int* col, double* E, double* grad_x,
                                   double* dE_dkappa, double* max_delta, void* stream);

/* Static text of a status code. */
const char* rcp_status_str(rcp_status s);

/* Message of the last failure on this handle ("" if none). */
const char* rcp_last_error(rcp_handle h);

#ifdef __cplusplus
}
#endif
#endif /* RCP_H */
