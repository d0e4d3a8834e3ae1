// rcp_kernels.cu -- per-iteration kernels of the binary64 path: initial
// positions, canonical tree reductions, the fused pair energy/gradient + Adam
// kernel, the kappa step with the stopping test, the standalone Adam step and
// shrink-to-contact.
//
// Every binary64 expression below is written in the exact order of the
// definition it implements (compiled with -fmad=false, so each operation
// rounds once, as IEEE-754 prescribes).  Sums follow one canonical order:
// per-row sums are left folds over the row's partners in ascending index,
// global sums are pairwise trees over the particle index, zero-padded to a
// power of two.  The result is therefore independent of the launch shape and
// of which non-overlapping pairs happen to be listed.
#include "rcp_internal.cuh"


// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output k of the stream seeded with
// `seed` is the variant-13 mix of seed + (k + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long k)
{
    unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Back into [0, L) after a step shorter than L.
__device__ __forceinline__ double wrap_step(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

// Minimum-image component of x_i - x_j.
__device__ __forceinline__ double min_image(double t, double L, double h)
{
    if (t > h) t = t - L;
    else if (t < -h) t = t + L;
    return t;
}

// Component a of x_i - x_j: minimum image on a periodic axis, the plain
// difference on an axis bounded by flat walls or the container (c.bounded).
__device__ __forceinline__ double axis_diff(const RcpConst& c, int a, double t)
{
    return ((c.bounded >> a) & 1) ? t : min_image(t, c.L[a], c.halfL[a]);
}

// Coordinate a after a step: wrapped on a periodic axis, kept on a bounded one.
__device__ __forceinline__ double axis_wrap(const RcpConst& c, int a, double x)
{
    return ((c.bounded >> a) & 1) ? x : wrap_step(x, c.L[a]);
}

// Distance from a sphere's centre to the container's centre (ball) or axis
// (cylinder), with the offsets x_a - L_a/2 over the container's axes (0 on
// the others); summed over the axes in order.
__device__ __forceinline__ double container_dist(const RcpConst& c, const double4_32a& xi, double off[3])
{
    double s2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double xa = a == 0 ? xi.x : (a == 1 ? xi.y : xi.z);
        off[a] = ((c.caxes >> a) & 1) ? xa - c.halfL[a] : 0.0;
        if ((c.caxes >> a) & 1) s2 = s2 + off[a] * off[a];
    }
    return sqrt(s2);
}

// Flat hard walls at 0 and L_a on every axis a whose bit is set in c.walls
// (Sec. II).  Sphere i (contact radius rad = kappa D^0/2, F/2 frozen) meets
// the wall at distance h when h < rad; with delta = 1 - h/rad its row takes
// eps/2 delta^2, eps delta (1 - delta)/kappa (mobile) and -+ eps delta / rad
// on dE/dx_a (mobile; the wall at 0 pushes towards +x_a).  Axes in order, the
// wall at 0 before the wall at L_a, after the row's pairs.
__device__ __forceinline__ void wall_terms(const RcpConst& c, double kappa, const double4_32a& xi, double& g0,
                                           double& g1, double& g2, double& e, double& k, double& md)
{
    const bool mob = xi.w > 0.0;
    const double rad = mob ? kappa * (0.5 * xi.w) : 0.5 * (-xi.w);
    for (int a = 0; a < 3; ++a) {
        if (!((c.walls >> a) & 1)) continue;
        const double xa = a == 0 ? xi.x : (a == 1 ? xi.y : xi.z);
        for (int side = 0; side < 2; ++side) {
            const double h = side == 0 ? xa : c.L[a] - xa;
            const double delta = 1.0 - h / rad;
            if (!(delta > 0.0)) continue;
            if (mob) {
                const double f = (c.eps * delta) / rad;
                double& ga = a == 0 ? g0 : (a == 1 ? g1 : g2);
                ga = side == 0 ? ga - f : ga + f;
                k = k + ((c.eps * delta) * (1.0 - delta)) / kappa;
            }
            e = e + (0.5 * c.eps) * (delta * delta);
            if (delta > md) md = delta;
        }
    }
    if (c.container) {
        // the curved wall: h = R - |x - c|, d h / d x_a = -(x_a - c_a) / |x - c|
        double off[3];
        const double rc = container_dist(c, xi, off);
        const double h = c.Rc - rc;
        const double delta = 1.0 - h / rad;
        if (delta > 0.0) {
            if (mob) {
                if (rc > 0.0) {
                    const double f = ((c.eps * delta) / rad) / rc;
                    if (c.caxes & 1) g0 = g0 + f * off[0];
                    if (c.caxes & 2) g1 = g1 + f * off[1];
                    if (c.caxes & 4) g2 = g2 + f * off[2];
                }
                k = k + ((c.eps * delta) * (1.0 - delta)) / kappa;
            }
            e = e + (0.5 * c.eps) * (delta * delta);
            if (delta > md) md = delta;
        }
    }
}

// Binary64 maximum overlap of the current binary64 positions over the
// listed pairs and the walls, the pairs in k_pair64's arithmetic (confirms a
// mixed path's binary32 stop candidate).
__global__ void __launch_bounds__(RCP_PAIR_THREADS)
k_maxdelta64(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const unsigned int* rowptr,
             const unsigned int* col)
{
    const double4_32a* x = ctl->parity ? xB : xA;
    const double kappa = ctl->kappa;
    const long long i = (long long)blockIdx.x * RCP_PAIR_THREADS + threadIdx.x;
    double md = 0.0;
    if (i < c.N) {
        const double4_32a xi = x[i];
        for (unsigned int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            const unsigned int j = col[t];
            if ((long long)j < i) continue;
            const double4_32a xj = x[j];
            const double dx = axis_diff(c, 0, xi.x - xj.x), dy = axis_diff(c, 1, xi.y - xj.y),
                         dz = axis_diff(c, 2, xi.z - xj.z);
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double dd = (xi.w > 0.0 && xj.w > 0.0) ? kappa * (0.5 * (xi.w + xj.w))
                                                         : 0.5 * (size_at(xi.w, kappa) + size_at(xj.w, kappa));
            if (r2 > (dd * dd) * RCP_NO_OVERLAP_MARGIN) continue;   // certainly delta <= 0
            const double r = sqrt(r2);
            const double delta = 1.0 - r / dd;
            if (delta > md) md = delta;
        }
        if (c.walls | c.container) {
            double g0 = 0.0, g1 = 0.0, g2 = 0.0, e = 0.0, k = 0.0;
            wall_terms(c, kappa, xi, g0, g1, g2, e, k, md);
        }
    }
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_down_sync(0xffffffffu, md, o));
    if ((threadIdx.x & 31) == 0 && md > 0.0) atomicMax(&ctl->md64_bits, dbits(md));
}

__global__ void k_init_positions(unsigned long long seed, long long N, RcpConst c, const double* D0, double4_32a* x)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double p[3];
    for (int a = 0; a < 3; ++a) {
        if (a >= c.dim) {   // d = 2: every disk in the plane z = L_z / 2
            p[a] = c.halfL[a];
            continue;
        }
        unsigned long long z = splitmix64_at(seed, (unsigned long long)(c.dim * i + a));
        double u = (double)(z >> 11) * 0x1.0p-53;
        p[a] = wrap_step(c.L[a] * u, c.L[a]);
    }
    x[i] = make_double4_32a(p[0], p[1], p[2], D0[i]);
}

// Non-overlapping placement, round r of size class k (random sequential
// addition by class): every sphere of the class not yet placed draws its
// candidate, SplitMix64 outputs 3 (r N + i) + a (round 0 = the uniform state
// above); rejection marks are cleared for the round.
__global__ void k_place_draw(unsigned long long seed, long long N, long long r, int k, RcpConst c, const double* D0,
                             const int* lvl, const unsigned char* placed, unsigned char* reject, double4_32a* x)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    reject[i] = 0;
    if (placed[i] || lvl[i] != k) return;
    double p[3];
    for (int a = 0; a < 3; ++a) {
        if (a >= c.dim) {
            p[a] = c.halfL[a];
            continue;
        }
        unsigned long long z = splitmix64_at(seed, (unsigned long long)(c.dim * (r * N + i) + a));
        double u = (double)(z >> 11) * 0x1.0p-53;
        p[a] = wrap_step(c.L[a] * u, c.L[a]);
    }
    x[i] = make_double4_32a(p[0], p[1], p[2], D0[i]);
}

// Keep the candidates of class k that nothing rejected; count the rest.
__global__ void k_place_accept(RcpCtl* ctl, long long N, int k, const int* lvl, unsigned char* placed,
                               const unsigned char* reject)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || placed[i] || lvl[i] != k) return;
    if (!reject[i]) placed[i] = 1;
    else atomicAdd(&ctl->pair_cursor, 1ull);
}

// ---------------------------------------------------------------------------
// Canonical tree of the values held by the threads of a block, in thread
// order: adjacent lanes first (shuffle offsets 1, 2, 4, 8, 16), then adjacent
// warps.  NT is a power of two.  The result is valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_tree(double v, double* sh)
{
    for (int o = 1; o < 32; o <<= 1) {
        double w = __shfl_down_sync(0xffffffffu, v, o);
        v = v + w;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        constexpr int W = NT / 32;
        for (int s = 1; s < W; s <<= 1)
            for (int k = 0; k + s < W; k += 2 * s) sh[k] = sh[k] + sh[k + s];
        r = sh[0];
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        r = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    }
    __syncthreads();
    return r;
}

// Terms D, D^3 = (D D) D, D^4 = (D D)(D D) of the moment sums, one tree of
// RCP_TREE consecutive terms per block.  A positive power takes the mobile
// spheres' D^0 (a frozen sphere's term is 0), a negative one the frozen
// spheres' fixed diameters F (a mobile sphere's term is 0).
__global__ void __launch_bounds__(RCP_TREE) k_tree_terms(const double* D0, long long N, int power, double* out)
{
    __shared__ double sh[32];
    long long i = (long long)blockIdx.x * RCP_TREE + threadIdx.x;
    double v = 0.0;
    if (i < N) {
        double D = power > 0 ? mobile_part(D0[i]) : mobile_part(-D0[i]);
        if (power < 0) power = -power;
        if (power == 1) v = D;
        else if (power == 2) v = D * D;
        else if (power == 3) v = (D * D) * D;
        else v = (D * D) * (D * D);
    }
    double s = block_tree<RCP_TREE>(v, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// One level of a tree sum: block b sums in[b*RCP_TREE .. +RCP_TREE) (zero
// padded).  Applied until one value is left, this realises the pairwise tree
// over the zero-padded sequence.
__global__ void __launch_bounds__(RCP_TREE) k_tree_pass(const double* in, long long n, double* out)
{
    __shared__ double sh[32];
    long long i = (long long)blockIdx.x * RCP_TREE + threadIdx.x;
    double s = block_tree<RCP_TREE>(i < n ? in[i] : 0.0, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RCP_TREE) k_tree_pass2(const double* ina, const double* inb, long long n,
                                                         double* outa, double* outb)
{
    __shared__ double sh[32];
    long long i = (long long)blockIdx.x * RCP_TREE + threadIdx.x;
    double sa = block_tree<RCP_TREE>(i < n ? ina[i] : 0.0, sh);
    double sb = block_tree<RCP_TREE>(i < n ? inb[i] : 0.0, sh);
    if (threadIdx.x == 0) {
        outa[blockIdx.x] = sa;
        outb[blockIdx.x] = sb;
    }
}

// kappa_0: the cube root of phi0 V / (pi/6 sum D^3) by 200 Newton steps
// y <- (2y + a/y^2)/3 from y = 1 (correctly rounded operations only, so the
// bits do not depend on a math library).
__global__ void k_kappa0(RcpCtl* ctl, double phi0, double V, int dim)
{
    if (dim == 2) {   // area fraction of disks: kappa^2 (pi/4) sum D^2 = phi0 A
        ctl->kappa = sqrt((phi0 * V) / ((RCP_PI / 4.0) * ctl->SD2));
        return;
    }
    double a = (phi0 * V) / ((RCP_PI / 6.0) * ctl->SD3);
    double y = 1.0;
    if (a > 0.0)
        for (int it = 0; it < 200; ++it) y = (2.0 * y + a / (y * y)) / 3.0;
    else
        y = 0.0;
    ctl->kappa = y;
}

__global__ void k_set_rung(RcpCtl* ctl, RcpConst c, double mu, double eta_x, double eta_k, double tol,
                           long long iter_limit, int final_rung)
{
    ctl->mu = mu;
    ctl->eta_x = eta_x;
    ctl->eta_k = eta_k;
    ctl->tol = tol;
    ctl->iter_limit = iter_limit;
    ctl->final_rung = final_rung;
    ctl->halted = ctl->iter >= iter_limit ? 1 : 0;
    ctl->verify = 0;
    ctl->loop_last_iter = -1;
    if (!c.canon) mix_fill(ctl, c);
}

__global__ void k_clear_halt(RcpCtl* ctl) { ctl->halted = 0; }

// End of a body pass of the graph's device-side loop: run the body again
// unless an iteration halted (rebuild due, iteration limit, stop, error).
// A pass that did not advance the iteration count also ends the loop, with
// RCP_ERR_TIMEOUT, so the loop is bounded by the iteration limit whatever
// happens (every pass that does not halt advances the count).
__global__ void k_loop_cond(RcpCtl* ctl, cudaGraphConditionalHandle hc)
{
    ctl->body_passes += 1;
    bool more = !ctl->halted;
    if (more && ctl->iter == ctl->loop_last_iter) {
        ctl->status = RCP_ERR_TIMEOUT;
        ctl->halted = 1;
        more = false;
    }
    ctl->loop_last_iter = ctl->iter;
    if (!more) cudaGraphSetConditional(hc, 0);
}

// Rung values of every packing of a batch before a replay (thread p = packing p).
__global__ void k_batch_set(const PackDev* P, const RungSet* rs, int B)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B) return;
    RcpCtl* ctl = P[p].ctl;
    const RungSet r = rs[p];
    if (!r.active) {
        ctl->halted = 1;
        return;
    }
    ctl->mu = r.mu;
    ctl->eta_x = r.eta_x;
    ctl->eta_k = r.eta_k;
    ctl->tol = r.tol;
    ctl->iter_limit = r.iter_limit;
    ctl->final_rung = r.final_rung;
    ctl->halted = ctl->iter >= r.iter_limit ? 1 : 0;
    ctl->verify = 0;
    mix_fill(ctl, P[p].c);
}

// The fields the batch driver needs from every packing, in one array.
__global__ void k_batch_status(const PackDev* P, BatchStat* out, int B)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B) return;
    const RcpCtl* c = P[p].ctl;
    BatchStat s;
    s.iter = c->iter;
    s.rebuilds = c->rebuilds;
    s.kappa = c->kappa;
    s.E = c->E;
    s.maxdelta = c->maxdelta;
    s.pairs = c->pairs;
    s.halted = c->halted;
    s.stopped = c->stopped;
    s.need_rebuild = c->need_rebuild;
    s.status = c->status;
    s.verify = c->verify;
    s.parity = c->parity;
    out[p] = s;
}

// Caller positions [N][3] -> (x, y, z, D0) records, wrapped into the box.
// Positions from a caller's [N][3] array (sphere order of the caller; perm,
// when not NULL, gives the caller's index of each internal sphere).
// ctl (when not NULL) picks the buffer holding the current positions on the
// device (x = xB when the parity is odd), so the host need not read it.
__global__ void k_set_positions(long long N, RcpConst c, const double* xin, const double* D0, double4_32a* x,
                                const unsigned int* perm, const RcpCtl* ctl, double4_32a* xB)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (ctl && ctl->parity) x = xB;
    const long long u = perm ? (long long)perm[i] : i;
    double p[3];
    for (int a = 0; a < 3; ++a) {
        if (a >= c.dim) {   // d = 2: the plane z = L_z / 2
            p[a] = c.halfL[a];
            continue;
        }
        double v = xin[c.dim * u + a];
        if ((c.bounded >> a) & 1) {   // bounded axis: the caller's coordinate as it is
            p[a] = v;
            continue;
        }
        if (v < 0.0 || v >= c.L[a]) v = v - c.L[a] * floor(v / c.L[a]);
        p[a] = wrap_step(v, c.L[a]);
    }
    x[i] = make_double4_32a(p[0], p[1], p[2], D0[i]);
}

__global__ void k_get_positions(long long N, RcpConst c, const double4_32a* x, double* out, const unsigned int* perm)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long u = perm ? (long long)perm[i] : i;
    double4_32a p = x[i];
    out[c.dim * u + 0] = p.x;
    out[c.dim * u + 1] = p.y;
    if (c.dim == 3) out[3 * u + 2] = p.z;
}

// Vectors between the caller's layout ([N][dim], caller order) and the
// internal one ([N][3], internal order; perm NULL: the same order).
// to_caller: out[perm[i]] = in[i], the z column dropped when dim = 2;
// otherwise out[i] = in[perm[i]], z = 0 when dim = 2.
__global__ void k_perm3(long long N, RcpConst c, const unsigned int* perm, const double* in, double* out,
                        int to_caller)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long u = perm ? (long long)perm[i] : i;
    const int dc = c.dim;
    if (to_caller) {
        for (int a = 0; a < dc; ++a) out[dc * u + a] = in[3 * i + a];
    } else {
        for (int a = 0; a < 3; ++a) out[3 * i + a] = a < dc ? in[dc * u + a] : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba 2015, Algorithm 1) on one coordinate, the bias products
// b1 = beta1^t and b2 = beta2^t already advanced to this step.
__device__ __forceinline__ double adam_coord(double p, double g, double& m, double& v, double eta,
                                             const RcpConst& c, double h1, double h2)
{
    const double c1 = 1.0 - c.beta1, c2 = 1.0 - c.beta2;
    m = c.beta1 * m + c1 * g;
    v = c.beta2 * v + c2 * (g * g);
    double mh = m / h1;
    double vh = v / h2;
    return p - (eta * mh) / (sqrt(vh) + c.adam_eps);
}

// Skin budget of sphere i (exact Verlet criterion).  A pair is listed iff its
// distance at the build was below kappa_b d0 + sigma_i + sigma_j; it stays
// non-overlapping while |dx_i| + |dx_j| + (kappa - kappa_b) d0 <= sigma_i +
// sigma_j, which holds if every sphere keeps
//   |x_i - x_i^b| + (kappa - kappa_b) D_i / 2 <= theta sigma_i   (theta <= 1).
// The displacement part is known here; what it leaves for kappa growth,
// b_i = 2 (theta sigma_i - |x_i - x_i^b|) / D_i, is reduced to its minimum
// (the kappa step compares kappa - kappa_b with it).  A negative b_i flags
// the rebuild directly.  Margins of 1e-9 cover rounding.
__device__ __forceinline__ void skin_budget64(RcpCtl* ctl, const RcpConst& c, double px, double py, double pz,
                                              double D0, double4_32a b, float& bud)
{
    double dx = axis_diff(c, 0, px - b.x);
    double dy = axis_diff(c, 1, py - b.y);
    double dz = axis_diff(c, 2, pz - b.z);
    const double disp = sqrt(dx * dx + dy * dy + dz * dz) * (1.0 + 1e-9);
    const double sig = c.skin_theta * (c.skin_s * ctl->kappa_b * D0 + ctl->sigma0) * (1.0 - 1e-9);
    const double bi = 2.0 * (sig - disp) / D0;
    if (!(bi >= 0.0)) atomicOr(&ctl->disp_flag, 1u);
    else bud = fminf(bud, __double2float_rd(bi * (1.0 - 1e-9)));
}

// Warp minimum of the budgets, one atomic per warp (non-negative binary32
// values order like their bit patterns).
__device__ __forceinline__ void push_budget(RcpCtl* ctl, float bud)
{
    for (int o = 16; o > 0; o >>= 1) bud = fminf(bud, __shfl_down_sync(0xffffffffu, bud, o));
    if ((threadIdx.x & 31) == 0 && bud < INFINITY) {
        const unsigned int bits = __float_as_uint(bud);
        if (bits < *(volatile unsigned int*)&ctl->kbud_bits) atomicMin(&ctl->kbud_bits, bits);
    }
}

// Does kappa_new still fit the minimum budget (the rebuild test closing an
// iteration or a standalone Adam step)?  Resets the budget for the next one.
__device__ __forceinline__ bool skin_exhausted(RcpCtl* ctl, double kappa_new)
{
    const float bud = __uint_as_float(ctl->kbud_bits);
    ctl->kbud_bits = RCP_KBUD_INF;
    return ctl->disp_flag || (kappa_new - ctl->kappa_b) * (1.0 + 1e-9) > (double)bud;
}

// ---------------------------------------------------------------------------
// Fused pair kernel, binary64.  One thread per sphere i (row of the full
// Verlet list, columns ascending).  For every listed j with
// delta = 1 - r/d > 0, d = kappa (D_i^0 + D_j^0)/2:
//   g_i    -= eps delta / (d r) (x_i - x_j)_mi          (if r > 0)
//   e_i    += eps/2 delta^2,  k_i += eps delta (1 - delta)/kappa   (j > i)
//   maxd    = max(maxd, delta)
// Then, in Adam mode, the Adam step of x_i written to the other position
// buffer (rows still gather the current one), plus the skin check; in grad
// mode g_i is written out.  e_i and k_i are summed per block by the
// canonical tree; maxd by an atomic max (order-free).
__device__ __forceinline__ void pair64_body(RcpCtl* ctl, const RcpConst& c, double4_32a* xA, double4_32a* xB,
                                            double* m, double* v, const unsigned int* rowptr, const unsigned int* col,
                                            const double4_32a* xb, double* part_e, double* part_k, int mode,
                                            double* g_out, unsigned int blk, const double* row_e = nullptr,
                                            const double* row_k = nullptr)
{
    __shared__ double sh[RCP_PAIR_THREADS / 32];
    if (ctl->halted) return;
    const int parity = ctl->parity;
    const double4_32a* __restrict__ xin = parity ? xB : xA;
    double4_32a* __restrict__ xout = parity ? xA : xB;
    const double kappa = ctl->kappa;
    const long long i = (long long)blk * RCP_PAIR_THREADS + threadIdx.x;
    double e = 0.0, k = 0.0, md = 0.0;
    float bud = INFINITY;
    if (i < c.N && c.long64 && rowptr[i + 1] - rowptr[i] > c.long_row) {
        // a long row: k_pair64_long evaluated it (and took its Adam step)
        e = row_e[i];
        k = row_k[i];
    } else if (i < c.N) {
        const double4_32a xi = xin[i];
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        const unsigned int t1 = rowptr[i + 1];
        for (unsigned int t = rowptr[i]; t < t1; ++t) {
            const unsigned int j = col[t];
            const double4_32a xj = xin[j];
            double dx = axis_diff(c, 0, xi.x - xj.x);
            double dy = axis_diff(c, 1, xi.y - xj.y);
            double dz = axis_diff(c, 2, xi.z - xj.z);
            double r2 = dx * dx + dy * dy + dz * dz;
            const bool both = xi.w > 0.0 && xj.w > 0.0;   // no frozen sphere in the pair
            double dd = both ? kappa * (0.5 * (xi.w + xj.w)) : 0.5 * (size_at(xi.w, kappa) + size_at(xj.w, kappa));
            if (r2 > (dd * dd) * RCP_NO_OVERLAP_MARGIN) continue;   // certainly delta <= 0: no square root, no division
            double r = sqrt(r2);
            double delta = 1.0 - r / dd;
            if (delta > 0.0) {
                if (r > 0.0 && xi.w > 0.0) {
                    double coef = (c.eps * delta) / (dd * r);
                    g0 = g0 - coef * dx;
                    g1 = g1 - coef * dy;
                    g2 = g2 - coef * dz;
                }
                if ((long long)j > i) {
                    e = e + (0.5 * c.eps) * (delta * delta);
                    if (both)
                        k = k + ((c.eps * delta) * (1.0 - delta)) / kappa;
                    else   // d d / d kappa = (mobile D_i^0 + mobile D_j^0) / 2
                        k = k + (((c.eps * delta) * (1.0 - delta)) * (0.5 * (mobile_part(xi.w) + mobile_part(xj.w)))) / dd;
                }
                if (delta > md) md = delta;
            }
        }
        if (c.walls | c.container) wall_terms(c, kappa, xi, g0, g1, g2, e, k, md);
        if (mode == RCP_MODE_ADAM && !(xi.w > 0.0)) {
            xout[i] = xi;   // frozen: position and moments stay
        } else if (mode == RCP_MODE_ADAM) {
            const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
            const double h1 = 1.0 - b1, h2 = 1.0 - b2;
            const double eta = ctl->eta_x;
            double m0 = m[3 * i], m1 = m[3 * i + 1], m2 = m[3 * i + 2];
            double v0 = v[3 * i], v1 = v[3 * i + 1], v2 = v[3 * i + 2];
            double p0 = axis_wrap(c, 0, adam_coord(xi.x, g0, m0, v0, eta, c, h1, h2));
            double p1 = axis_wrap(c, 1, adam_coord(xi.y, g1, m1, v1, eta, c, h1, h2));
            double p2 = axis_wrap(c, 2, adam_coord(xi.z, g2, m2, v2, eta, c, h1, h2));
            m[3 * i] = m0; m[3 * i + 1] = m1; m[3 * i + 2] = m2;
            v[3 * i] = v0; v[3 * i + 1] = v1; v[3 * i + 2] = v2;
            xout[i] = make_double4_32a(p0, p1, p2, xi.w);
            skin_budget64(ctl, c, p0, p1, p2, xi.w, xb[i], bud);
        } else {
            g_out[3 * i] = g0;
            g_out[3 * i + 1] = g1;
            g_out[3 * i + 2] = g2;
        }
    }
    if (mode == RCP_MODE_ADAM) push_budget(ctl, bud);
    double se = block_tree<RCP_PAIR_THREADS>(e, sh);
    double sk = block_tree<RCP_PAIR_THREADS>(k, sh);
    double bm = block_max(md, sh);
    if (threadIdx.x == 0) {
        part_e[blk] = se;
        part_k[blk] = sk;
        if (bm > 0.0) atomicMax(&ctl->maxdelta_bits, dbits(bm));
    }
}

__global__ void __launch_bounds__(RCP_PAIR_THREADS)
k_pair64(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
         const unsigned int* rowptr, const unsigned int* col, const double4_32a* xb,
         double* part_e, double* part_k, int mode, double* g_out, const double* row_e, const double* row_k)
{
    pair64_body(ctl, c, xA, xB, m, v, rowptr, col, xb, part_e, part_k, mode, g_out, blockIdx.x, row_e, row_k);
}

// Binary64 pair kernel for small N: one warp per row.  With a thread per
// row, a small packing occupies a few SMs while each thread walks its row
// through a serial chain of binary64 square roots and divisions (slow on
// B300).  Here the lanes compute the terms of up to 32 partners at once and
// lane 0 folds them in the row's order -- the same products and the same
// left folds as pair64_body, so the sums are bit-identical -- then the wall
// terms.  e_i and k_i go to row_e/row_k[i] for the canonical tree over the
// rows; lanes 0-2 take the Adam step of one coordinate each.
// One row of the binary64 pair kernel by a whole warp: the lanes compute the
// terms of up to 32 partners at once, lane 0's order folds them (the row's
// order: the same products and the same left folds as pair64_body, so the
// sums are bit-identical), then the wall terms; e_i and k_i go to
// row_e/row_k[i]; lanes 0-2 take the Adam step of one coordinate each.
__device__ __forceinline__ void warp_row64(RcpCtl* ctl, const RcpConst& c, const double4_32a* __restrict__ xin,
                                           double4_32a* __restrict__ xout, double* m, double* v,
                                           const unsigned int* rowptr, const unsigned int* col,
                                           const double4_32a* xb, double* row_e, double* row_k, int mode,
                                           double* g_out, long long i, int lane, double kappa, double& md,
                                           float& bud)
{
    const unsigned int FULL = 0xffffffffu;
    {
        const double4_32a xi = xin[i];
        double g0 = 0.0, g1 = 0.0, g2 = 0.0, e = 0.0, k = 0.0;   // the fold, the same in every lane
        const unsigned int t0 = rowptr[i], t1 = rowptr[i + 1];
        for (unsigned int base = t0; base < t1; base += 32) {
            const unsigned int t = base + (unsigned int)lane;
            bool hit = false, grad = false, upper = false;
            double tx = 0.0, ty = 0.0, tz = 0.0, te = 0.0, tk = 0.0;
            if (t < t1) {
                const unsigned int j = col[t];
                const double4_32a xj = xin[j];
                double dx = axis_diff(c, 0, xi.x - xj.x);
                double dy = axis_diff(c, 1, xi.y - xj.y);
                double dz = axis_diff(c, 2, xi.z - xj.z);
                double r2 = dx * dx + dy * dy + dz * dz;
                const bool both = xi.w > 0.0 && xj.w > 0.0;
                double dd = both ? kappa * (0.5 * (xi.w + xj.w)) : 0.5 * (size_at(xi.w, kappa) + size_at(xj.w, kappa));
                double delta = 0.0;
                if (!(r2 > (dd * dd) * RCP_NO_OVERLAP_MARGIN)) {   // else certainly delta <= 0
                    double r = sqrt(r2);
                    delta = 1.0 - r / dd;
                    if (delta > 0.0 && r > 0.0 && xi.w > 0.0) {
                        grad = true;
                        double coef = (c.eps * delta) / (dd * r);
                        tx = coef * dx;
                        ty = coef * dy;
                        tz = coef * dz;
                    }
                }
                if (delta > 0.0) {
                    hit = true;
                    if ((long long)j > i) {
                        upper = true;
                        te = (0.5 * c.eps) * (delta * delta);
                        if (both)
                            tk = ((c.eps * delta) * (1.0 - delta)) / kappa;
                        else
                            tk = (((c.eps * delta) * (1.0 - delta)) * (0.5 * (mobile_part(xi.w) + mobile_part(xj.w)))) / dd;
                    }
                    if (delta > md) md = delta;
                }
            }
            const unsigned int gm = __ballot_sync(FULL, grad), um = __ballot_sync(FULL, upper);
            unsigned int hm = __ballot_sync(FULL, hit);
            while (hm) {   // partners in the row's order (lowest lane first)
                const int l = __ffs(hm) - 1;
                hm &= hm - 1;
                const double ax = __shfl_sync(FULL, tx, l), ay = __shfl_sync(FULL, ty, l);
                const double az = __shfl_sync(FULL, tz, l), ae = __shfl_sync(FULL, te, l);
                const double ak = __shfl_sync(FULL, tk, l);
                if ((gm >> l) & 1u) {
                    g0 = g0 - ax;
                    g1 = g1 - ay;
                    g2 = g2 - az;
                }
                if ((um >> l) & 1u) {
                    e = e + ae;
                    k = k + ak;
                }
            }
        }
        if (c.walls | c.container) wall_terms(c, kappa, xi, g0, g1, g2, e, k, md);   // identical in every lane
        if (lane == 0) {
            row_e[i] = e;
            row_k[i] = k;
        }
        if (mode == RCP_MODE_ADAM && !(xi.w > 0.0)) {
            if (lane == 0) xout[i] = xi;   // frozen: position and moments stay
        } else if (mode == RCP_MODE_ADAM) {
            const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
            const double h1 = 1.0 - b1, h2 = 1.0 - b2;
            const double eta = ctl->eta_x;
            double pa = 0.0;
            if (lane < 3) {
                const double ga = lane == 0 ? g0 : (lane == 1 ? g1 : g2);
                const double xa = lane == 0 ? xi.x : (lane == 1 ? xi.y : xi.z);
                double ma = m[3 * i + lane], va = v[3 * i + lane];
                pa = axis_wrap(c, lane, adam_coord(xa, ga, ma, va, eta, c, h1, h2));
                m[3 * i + lane] = ma;
                v[3 * i + lane] = va;
            }
            const double p0 = __shfl_sync(FULL, pa, 0), p1 = __shfl_sync(FULL, pa, 1), p2 = __shfl_sync(FULL, pa, 2);
            if (lane == 0) {
                xout[i] = make_double4_32a(p0, p1, p2, xi.w);
                skin_budget64(ctl, c, p0, p1, p2, xi.w, xb[i], bud);
            }
        } else if (lane == 0) {
            g_out[3 * i] = g0;
            g_out[3 * i + 1] = g1;
            g_out[3 * i + 2] = g2;
        }
    }
}

__global__ void __launch_bounds__(RCP_WARP_ROW_THREADS)
k_pair64_warp(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
              const unsigned int* rowptr, const unsigned int* col, const double4_32a* xb, double* row_e,
              double* row_k, int mode, double* g_out)
{
    __shared__ double sh[RCP_WARP_ROW_THREADS / 32];
    if (ctl->halted) return;
    const int lane = threadIdx.x & 31;
    const int parity = ctl->parity;
    const double4_32a* __restrict__ xin = parity ? xB : xA;
    double4_32a* __restrict__ xout = parity ? xA : xB;
    const long long i = ((long long)blockIdx.x * RCP_WARP_ROW_THREADS + threadIdx.x) >> 5;   // warp-uniform
    double md = 0.0;
    float bud = INFINITY;
    if (i < c.N)
        warp_row64(ctl, c, xin, xout, m, v, rowptr, col, xb, row_e, row_k, mode, g_out, i, lane, ctl->kappa, md,
                   bud);
    if (mode == RCP_MODE_ADAM) push_budget(ctl, bud);
    const double bm = block_max(md, sh);
    if (threadIdx.x == 0 && bm > 0.0) atomicMax(&ctl->maxdelta_bits, dbits(bm));
}

// The rows longer than c.long_row of a large binary64 packing, a warp each
// (launched before k_pair64, which then takes their e_i, k_i from row_e /
// row_k for its block trees): with one thread per row, the few rows of the
// largest spheres (thousands of entries at S = 5e5) would run on long after
// every other row has finished.
__global__ void __launch_bounds__(RCP_PAIR_THREADS)
k_pair64_long(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
              const unsigned int* rowptr, const unsigned int* col, const unsigned int* long_rows,
              const double4_32a* xb, double* row_e, double* row_k, int mode, double* g_out)
{
    __shared__ double sh[RCP_PAIR_THREADS / 32];
    if (ctl->halted) return;
    const int lane = threadIdx.x & 31;
    const int parity = ctl->parity;
    const double4_32a* __restrict__ xin = parity ? xB : xA;
    double4_32a* __restrict__ xout = parity ? xA : xB;
    const double kappa = ctl->kappa;
    const unsigned int nlong = ctl->n_long;
    const unsigned int nw = gridDim.x * (RCP_PAIR_THREADS / 32);
    double md = 0.0;
    float bud = INFINITY;
    for (unsigned int r = blockIdx.x * (RCP_PAIR_THREADS / 32) + (threadIdx.x >> 5); r < nlong; r += nw)
        warp_row64(ctl, c, xin, xout, m, v, rowptr, col, xb, row_e, row_k, mode, g_out, (long long)long_rows[r],
                   lane, kappa, md, bud);
    if (mode == RCP_MODE_ADAM) push_budget(ctl, bud);
    const double bm = block_max(md, sh);
    if (threadIdx.x == 0 && bm > 0.0) atomicMax(&ctl->maxdelta_bits, dbits(bm));
}

// Packing of a block in a batched launch: the last p with bstart[p] <= block.
__device__ __forceinline__ int batch_pack(const unsigned int* bstart, int B, unsigned int block)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bstart[mid] <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched binary64 pair kernel: block b serves packing p = batch_pack(b)
// with local block b - bstart[p], so each packing computes exactly what its
// own launch would.
__global__ void __launch_bounds__(RCP_PAIR_THREADS) k_pair64_batch(const PackDev* P, const unsigned int* bstart,
                                                                   int B, int mode)
{
    const int p = batch_pack(bstart, B, blockIdx.x);
    const PackDev& q = P[p];
    pair64_body(q.ctl, q.c, q.xA, q.xB, q.m64, q.v64, q.rowptr, q.col, q.xb, q.part_e, q.part_k, mode, q.g,
                blockIdx.x - bstart[p]);
}

// Close an iteration: Adam step of kappa with dE/dkappa of the evaluation,
// advance the bias products, swap the position buffers, count the step, and
// flag a rebuild when some sphere used up theta of its skin or kappa grew
// past kappa_b (1 + 2 s (1 - theta)).
__device__ void kappa_adam_tail(RcpCtl* ctl, const RcpConst& c)
{
    const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
    double mk = ctl->mk, vk = ctl->vk;
    const double kn = adam_coord(ctl->kappa, ctl->dEdk, mk, vk, ctl->eta_k, c, 1.0 - b1, 1.0 - b2);
    ctl->mk = mk;
    ctl->vk = vk;
    ctl->kappa = kn;
    ctl->b1 = b1;
    ctl->b2 = b2;
    ctl->parity ^= 1;
    ctl->iter += 1;
    if (ctl->iter >= ctl->iter_limit) ctl->halted = 1;
    if (skin_exhausted(ctl, kn)) {
        ctl->need_rebuild = 1;
        ctl->halted = 1;
    }
    if (!c.canon) mix_fill(ctl, c);
}

// ---------------------------------------------------------------------------
// Finish an evaluation: tree over the block partials (nb <= 8192, zero
// padded to a power of two) gives sum_i e_i and sum_i k_i, hence
//   E = sum e - mu (kappa sum D^0),   dE/dkappa = sum k - mu sum D^0.
// In Adam mode: the stopping test of App. A on the state just evaluated (the
// final rung stops when max delta < tol, before that state's Adam step),
// otherwise the Adam step of kappa, the buffer swap, and the rebuild test.
__device__ __forceinline__ void kappa_step_body(RcpCtl* ctl, const RcpConst& c, const double* part_e,
                                                const double* part_k, long long nb, int mode, double* buf)
{
    if (ctl->halted) return;
    long long M = 1;
    while (M < nb) M <<= 1;
    double* be = buf;
    double* bk = buf + M;
    for (long long t = threadIdx.x; t < M; t += blockDim.x) {
        be[t] = t < nb ? part_e[t] : 0.0;
        bk[t] = t < nb ? part_k[t] : 0.0;
    }
    __syncthreads();
    for (long long s = 1; s < M; s <<= 1) {
        for (long long idx = (long long)threadIdx.x * 2 * s; idx < M; idx += (long long)blockDim.x * 2 * s) {
            be[idx] = be[idx] + be[idx + s];
            bk[idx] = bk[idx] + bk[idx + s];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    kappa_close(ctl, c, be[0], bk[0], mode);
}

// The scalar part of closing an evaluation (one thread), from the sums of the
// pair terms: E and dE/dkappa with the growth term, the largest overlap, the
// stopping test of App. A, and in Adam mode the kappa step.
__device__ void kappa_close(RcpCtl* ctl, const RcpConst& c, double se, double sk, int mode)
{
    const double mu = ctl->mu, kappa = ctl->kappa;
    const double E = se - mu * (kappa * ctl->SD);
    const double dEdk = sk - mu * ctl->SD;
    const double md = bitsd(ctl->maxdelta_bits);
    ctl->maxdelta_bits = 0ull;
    ctl->E = E;
    ctl->dEdk = dEdk;
    ctl->maxdelta = md;
    if (!isfinite(E) || !isfinite(dEdk)) {
        ctl->status = RCP_ERR_NAN;
        ctl->halted = 1;
        return;
    }
    if (mode != RCP_MODE_ADAM) return;
    if (ctl->final_rung) {
        if (c.stop_margin == 0.0) {
            if (md < ctl->tol) {
                ctl->stopped = 1;
                ctl->halted = 1;
                return;
            }
        } else if (md < ctl->tol * (1.0 + c.stop_margin)) {
            // binary32 overlaps: a stop candidate is confirmed in binary64
            // (k_maxdelta64, k_verify_final) before the iteration is closed
            ctl->verify = 1;
            ctl->halted = 1;
            return;
        }
    }
    kappa_adam_tail(ctl, c);
}

__global__ void __launch_bounds__(1024) k_kappa_step(RcpCtl* ctl, RcpConst c, const double* part_e,
                                                     const double* part_k, long long nb, int mode)
{
    extern __shared__ double buf[];
    kappa_step_body(ctl, c, part_e, part_k, nb, mode, buf);
}

// Batched kappa step: block p closes the iteration of packing p.
__global__ void __launch_bounds__(1024) k_kappa_step_batch(const PackDev* P, int mode)
{
    extern __shared__ double buf[];
    const PackDev& q = P[blockIdx.x];
    kappa_step_body(q.ctl, q.c, q.part_e, q.part_k, q.nparts, mode, buf);
}

// Close a mixed-precision evaluation: the block partials (compensated binary32
// pairs, one per block of the pair kernel) are summed in one fixed order -- thread t takes partials t, t + 1024,
// ... with 2Sum, then the threads' pairs meet in a fixed tree -- and widened to
// binary64 at the end (binary64 adds are slow on B300, and the partials carry
// no more than binary32 pairs anyway); the rest is the kappa step of the
// binary64 path.  One kernel instead of a tree pass and the kappa step.
__device__ __forceinline__ void kappa_mixed_body(RcpCtl* ctl, const RcpConst& c, const float2* pe, const float2* pk,
                                                 long long n, int mode)
{
    __shared__ float sh[4][32];
    if (ctl->halted) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float es = 0.f, ec = 0.f, ks = 0.f, kc = 0.f;
    for (long long t = tid; t < n; t += blockDim.x) {
        const float2 a = pe[t], b = pk[t];
        acc2(es, ec, a.x);
        ec = ec + a.y;
        acc2(ks, kc, b.x);
        kc = kc + b.y;
    }
    warp_sum2(es, ec);
    warp_sum2(ks, kc);
    if (lane == 0) {
        sh[0][warp] = es;
        sh[1][warp] = ec;
        sh[2][warp] = ks;
        sh[3][warp] = kc;
    }
    __syncthreads();
    if (warp != 0) return;
    const int nw = (int)(blockDim.x >> 5);
    es = lane < nw ? sh[0][lane] : 0.f;
    ec = lane < nw ? sh[1][lane] : 0.f;
    ks = lane < nw ? sh[2][lane] : 0.f;
    kc = lane < nw ? sh[3][lane] : 0.f;
    warp_sum2(es, ec);
    warp_sum2(ks, kc);
    if (lane == 0) kappa_close(ctl, c, (double)es + (double)ec, (double)ks + (double)kc, mode);
}

__global__ void __launch_bounds__(1024) k_kappa_mixed(RcpCtl* ctl, RcpConst c, const double* part_e,
                                                      const double* part_k, long long n, int mode)
{
    kappa_mixed_body(ctl, c, reinterpret_cast<const float2*>(part_e), reinterpret_cast<const float2*>(part_k), n,
                     mode);
}

// Batched: block p closes the iteration of packing p.
__global__ void __launch_bounds__(1024) k_kappa_mixed_batch(const PackDev* P, int mode)
{
    const PackDev& q = P[blockIdx.x];
    kappa_mixed_body(q.ctl, q.c, reinterpret_cast<const float2*>(q.part_e), reinterpret_cast<const float2*>(q.part_k),
                     q.nparts, mode);
}

// Binary64 verdict on a binary32 stop candidate: stop on the evaluated state,
// or close the iteration as k_kappa_step would have.
__global__ void k_verify_final(RcpCtl* ctl, RcpConst c)
{
    const double md = bitsd(ctl->md64_bits);
    ctl->md64_bits = 0ull;
    ctl->verify = 0;
    if (md < ctl->tol) {
        ctl->maxdelta = md;
        ctl->stopped = 1;
        ctl->halted = 1;
        return;
    }
    ctl->halted = 0;
    kappa_adam_tail(ctl, c);
}

// ---------------------------------------------------------------------------
// Standalone Adam step on every coordinate (rcp_adam_step), in place on the
// current buffer, with a caller-supplied gradient [N][3].
__global__ void k_adam64(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
                         const double* g, const double4_32a* xb, double eta_x)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float bud = INFINITY;
    if (i < c.N && (ctl->parity ? xB : xA)[i].w > 0.0) {   // frozen spheres stay
        double4_32a* x = ctl->parity ? xB : xA;
        const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
        const double h1 = 1.0 - b1, h2 = 1.0 - b2;
        double4_32a p = x[i];
        double m0 = m[3 * i], m1 = m[3 * i + 1], m2 = m[3 * i + 2];
        double v0 = v[3 * i], v1 = v[3 * i + 1], v2 = v[3 * i + 2];
        double p0 = axis_wrap(c, 0, adam_coord(p.x, g[3 * i], m0, v0, eta_x, c, h1, h2));
        double p1 = axis_wrap(c, 1, adam_coord(p.y, g[3 * i + 1], m1, v1, eta_x, c, h1, h2));
        double p2 = axis_wrap(c, 2, adam_coord(p.z, g[3 * i + 2], m2, v2, eta_x, c, h1, h2));
        m[3 * i] = m0; m[3 * i + 1] = m1; m[3 * i + 2] = m2;
        v[3 * i] = v0; v[3 * i + 1] = v1; v[3 * i + 2] = v2;
        x[i] = make_double4_32a(p0, p1, p2, p.w);
        skin_budget64(ctl, c, p0, p1, p2, p.w, xb[i], bud);
    }
    push_budget(ctl, bud);
}

// kappa's share of the standalone Adam step; also advances t and the bias
// products, and flags a rebuild if the skin budget is used up.
__global__ void k_adam_kappa(RcpCtl* ctl, RcpConst c, double dEdk, double eta_k)
{
    const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
    double mk = ctl->mk, vk = ctl->vk;
    const double kn = adam_coord(ctl->kappa, dEdk, mk, vk, eta_k, c, 1.0 - b1, 1.0 - b2);
    ctl->mk = mk;
    ctl->vk = vk;
    ctl->kappa = kn;
    ctl->b1 = b1;
    ctl->b2 = b2;
    ctl->iter += 1;
    if (skin_exhausted(ctl, kn)) ctl->need_rebuild = 1;
    if (!c.canon) mix_fill(ctl, c);
}

// Skin check of the current state against the last build (after positions or
// kappa were replaced from outside): a sphere's displacement plus its share of
// kappa - kappa_b must stay within theta of its skin.
__global__ void k_disp_check(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                             const double4_32a* xb)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double4_32a* x = ctl->parity ? xB : xA;
    const double4_32a p = x[i], b = xb[i];
    if (!(p.w > 0.0)) return;   // a frozen sphere neither moves nor grows
    double dx = axis_diff(c, 0, p.x - b.x);
    double dy = axis_diff(c, 1, p.y - b.y);
    double dz = axis_diff(c, 2, p.z - b.z);
    const double disp = sqrt(dx * dx + dy * dy + dz * dz) * (1.0 + 1e-9);
    const double sig = c.skin_theta * (c.skin_s * ctl->kappa_b * p.w + ctl->sigma0) * (1.0 - 1e-9);
    if (disp + (ctl->kappa - ctl->kappa_b) * p.w * 0.5 * (1.0 + 1e-9) > sig) ctl->need_rebuild = 1;
}

// ---------------------------------------------------------------------------
// Shrink to contact: min over listed pairs i < j of r_ij / d_ij^0 (order-free
// minimum through the bit pattern of a non-negative double).  A pair with one
// frozen sphere (diameter F) touches at kappa = (r - F/2) / (D_a^0 / 2),
// lowered by (1 - 2^-40) for the bits the subtraction may cancel and clamped
// at 0; two frozen spheres set no bound.
__global__ void __launch_bounds__(RCP_PAIR_THREADS)
k_shrink(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
         const unsigned int* rowptr, const unsigned int* col)
{
    __shared__ double sh[RCP_PAIR_THREADS / 32];
    const double4_32a* x = ctl->parity ? xB : xA;
    const long long i = (long long)blockIdx.x * RCP_PAIR_THREADS + threadIdx.x;
    double q = INFINITY;
    if (i < c.N) {
        const double4_32a xi = x[i];
        for (unsigned int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            const unsigned int j = col[t];
            if ((long long)j <= i) continue;
            const double4_32a xj = x[j];
            double dx = axis_diff(c, 0, xi.x - xj.x);
            double dy = axis_diff(c, 1, xi.y - xj.y);
            double dz = axis_diff(c, 2, xi.z - xj.z);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double qq;
            if (xi.w > 0.0 && xj.w > 0.0) {
                qq = r / (0.5 * (xi.w + xj.w));
            } else if (xi.w > 0.0 || xj.w > 0.0) {
                const double Da = xi.w > 0.0 ? xi.w : xj.w;
                const double F = xi.w > 0.0 ? -xj.w : -xi.w;
                qq = ((r - 0.5 * F) / (0.5 * Da)) * (1.0 - 0x1.0p-40);
                if (qq < 0.0) qq = 0.0;
            } else {
                continue;
            }
            if (qq < q) q = qq;
        }
        if ((c.walls | c.container) && xi.w > 0.0) {   // a mobile sphere touches a wall at kappa = 2h / D^0
            if (c.container) {
                double off[3];
                const double h = c.Rc - container_dist(c, xi, off);
                double qq = (2.0 * h) / xi.w;
                if (qq < 0.0) qq = 0.0;
                if (qq < q) q = qq;
            }
            for (int a = 0; a < 3; ++a) {
                if (!((c.walls >> a) & 1)) continue;
                const double xa = a == 0 ? xi.x : (a == 1 ? xi.y : xi.z);
                for (int side = 0; side < 2; ++side) {
                    const double h = side == 0 ? xa : c.L[a] - xa;
                    double qq = (2.0 * h) / xi.w;
                    if (qq < 0.0) qq = 0.0;
                    if (qq < q) q = qq;
                }
            }
        }
    }
    // block minimum through max of the negated value
    double bm = -block_max(-q, sh);
    if (threadIdx.x == 0 && bm < INFINITY) atomicMin(&ctl->shrink_bits, dbits(bm));
}

// kappa_c = min(kappa, q_min) (1 - 2^-50): lowered by a few units in the
// last place so that no pair overlaps when re-evaluated in binary64;
// phi = ((pi/6) kappa_c^3 sum D^3 + (pi/6) sum_frozen F^3) / V.
__global__ void k_shrink_final(RcpCtl* ctl, RcpConst c)
{
    double q = bitsd(ctl->shrink_bits);
    double kc = ctl->kappa;
    if (q < kc) kc = q;
    kc = kc * (1.0 - 0x1.0p-50);
    ctl->kappa_c = kc;
    if (c.dim == 2) ctl->phi = ((((RCP_PI / 4.0) * (kc * kc)) * ctl->SD2) + (RCP_PI / 4.0) * ctl->SF2) / c.Vs;
    else ctl->phi = ((((RCP_PI / 6.0) * ((kc * kc) * kc)) * ctl->SD3) + (RCP_PI / 6.0) * ctl->SF3) / c.Vs;
}
