// rcp_mixed.cu -- the mixed-precision pair kernel.
//
// Positions stay binary64 (the optimiser's state) and each sphere also keeps a
// 32-byte pair record: a 32-bit fixed-point position q_a = floor(x_a / L_a
// 2^32) per axis, the binary32 remainder l_a = x_a / L_a 2^32 - q_a, and
// D_i^0.  The displacement of a pair is (q_i - q_j) in 32-bit integer
// arithmetic -- the wrap-around of the subtraction is exactly the periodic
// minimum image -- plus (l_i - l_j), scaled to length by L_a 2^-32, so every
// pair's separation is formed to binary32 relative precision at any scale
// (from the largest spheres down to D_max / 5e5).  Distance, overlap and the
// pair terms are binary32; each row sums them with a compensated (2Sum)
// accumulation, the row sums are widened to binary64 for the global trees,
// and the Adam moments are binary32 while the position update is binary64.
// The stopping test of App. A is confirmed in binary64 (k_maxdelta64).
#include "rcp_internal.cuh"

__device__ __forceinline__ void to_fixed(double x, double L, int& q, float& l)
{
    double t = (x / L) * 4294967296.0;
    double f = floor(t);
    q = (int)(unsigned int)(unsigned long long)f;  // x == L would give 2^32, i.e. 0
    l = (float)(t - f);
}

__device__ __forceinline__ MixRec make_rec(double4_32a p, const RcpConst& c)
{
    MixRec r;
    to_fixed(p.x, c.L[0], r.q.x, r.l.x);
    to_fixed(p.y, c.L[1], r.q.y, r.l.y);
    to_fixed(p.z, c.L[2], r.q.z, r.l.z);
    r.q.w = 0;
    r.l.w = (float)p.w;
    return r;
}

// Displacement a - b of two records along one axis, in length units.
__device__ __forceinline__ float rec_dx(int qa, float la, int qb, float lb, float scale)
{
    const int dq = (int)((unsigned int)qa - (unsigned int)qb);
    return ((float)dq + (la - lb)) * scale;
}

// Records of the current positions, and the build snapshot when rb != NULL.
__global__ void k_to_fixed(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, MixRec* rA, MixRec* rB,
                           MixRec* rb)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const int parity = ctl->parity;
    const MixRec r = make_rec((parity ? xB : xA)[i], c);
    (parity ? rB : rA)[i] = r;
    if (rb) rb[i] = r;
}

// 2Sum accumulation: s + c carries the exact sum of the added binary32 terms
// to within one rounding of the final value (Knuth's TwoSum, no FMA).
__device__ __forceinline__ void acc2(float& s, float& c, float x)
{
    const float t = s + x;
    const float z = t - s;
    c = c + ((s - (t - z)) + (x - z));
    s = t;
}

__device__ __forceinline__ double block_tree256(double v, double* sh)
{
    for (int o = 1; o < 32; o <<= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int s = 1; s < RCP_PAIR_THREADS / 32; s <<= 1)
            for (int k = 0; k + s < RCP_PAIR_THREADS / 32; k += 2 * s) sh[k] = sh[k] + sh[k + s];
        r = sh[0];
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ float warp_maxf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// One thread per sphere i (row of the full list).  Same terms as k_pair64,
// in binary32 on fixed-point displacements.
__global__ void __launch_bounds__(RCP_PAIR_THREADS)
k_pair_mixed(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, float* m, float* v, MixRec* rA, MixRec* rB,
             const unsigned int* rowptr, const unsigned int* col, const MixRec* rb, double* part_e, double* part_k,
             int mode, double* g_out)
{
    __shared__ double sh[RCP_PAIR_THREADS / 32];
    __shared__ float shm[RCP_PAIR_THREADS / 32];
    if (ctl->halted) return;
    const int parity = ctl->parity;
    const MixRec* __restrict__ rin = parity ? rB : rA;
    MixRec* __restrict__ rout = parity ? rA : rB;
    const double kappa = ctl->kappa;
    const float kf = (float)kappa;
    const float epsf = (float)c.eps;
    const float sx = c.qscale[0], sy = c.qscale[1], sz = c.qscale[2];
    const long long i = (long long)blockIdx.x * RCP_PAIR_THREADS + threadIdx.x;
    float es = 0.f, ec = 0.f, ks = 0.f, kc = 0.f, md = 0.f;
    if (i < c.N) {
        const MixRec ri = rin[i];
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
        const unsigned int t1 = rowptr[i + 1];
        for (unsigned int t = rowptr[i]; t < t1; ++t) {
            const unsigned int j = col[t];
            const MixRec rj = rin[j];
            const float dx = rec_dx(ri.q.x, ri.l.x, rj.q.x, rj.l.x, sx);
            const float dy = rec_dx(ri.q.y, ri.l.y, rj.q.y, rj.l.y, sy);
            const float dz = rec_dx(ri.q.z, ri.l.z, rj.q.z, rj.l.z, sz);
            const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
            const float r = sqrtf(r2);
            const float dd = kf * (0.5f * (ri.l.w + rj.l.w));
            const float delta = 1.0f - r / dd;
            if (delta > 0.0f) {
                if (r > 0.0f) {
                    const float coef = (epsf * delta) / (dd * r);
                    acc2(g0, c0, -coef * dx);
                    acc2(g1, c1, -coef * dy);
                    acc2(g2, c2, -coef * dz);
                }
                if ((long long)j > i) {
                    acc2(es, ec, (0.5f * epsf) * (delta * delta));
                    acc2(ks, kc, ((epsf * delta) * (1.0f - delta)) / kf);
                }
                md = fmaxf(md, delta);
            }
        }
        g0 = g0 + c0;
        g1 = g1 + c1;
        g2 = g2 + c2;
        if (mode == RCP_MODE_ADAM) {
            const double4_32a* xin = parity ? xB : xA;
            double4_32a* xout = parity ? xA : xB;
            const double4_32a xi = xin[i];
            const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
            const float h1 = (float)(1.0 - b1), h2 = (float)(1.0 - b2);
            const float be1 = (float)c.beta1, be2 = (float)c.beta2;
            const float o1 = (float)(1.0 - c.beta1), o2 = (float)(1.0 - c.beta2);
            const float etaf = (float)ctl->eta_x, aeps = (float)c.adam_eps;
            float gg[3] = {g0, g1, g2};
            double p[3] = {xi.x, xi.y, xi.z};
            for (int a = 0; a < 3; ++a) {
                float mm = be1 * m[3 * i + a] + o1 * gg[a];
                float vv = be2 * v[3 * i + a] + o2 * (gg[a] * gg[a]);
                m[3 * i + a] = mm;
                v[3 * i + a] = vv;
                const float step = (etaf * (mm / h1)) / (sqrtf(vv / h2) + aeps);
                double q = p[a] - (double)step;
                if (q < 0.0) q = q + c.L[a];
                if (q >= c.L[a]) q = q - c.L[a];
                p[a] = q;
            }
            const double4_32a xn = make_double4_32a(p[0], p[1], p[2], xi.w);
            xout[i] = xn;
            const MixRec rn = make_rec(xn, c);
            rout[i] = rn;
            // skin check against the build snapshot, binary32 with a margin
            const MixRec b = rb[i];
            const float ex = rec_dx(rn.q.x, rn.l.x, b.q.x, b.l.x, sx);
            const float ey = rec_dx(rn.q.y, rn.l.y, b.q.y, b.l.y, sy);
            const float ez = rec_dx(rn.q.z, rn.l.z, b.q.z, b.l.z, sz);
            const float lim = (float)(c.skin_theta * (c.skin_s * ctl->kappa_b * xi.w + ctl->sigma0) * (1.0 - 1e-5));
            if (ex * ex + ey * ey + ez * ez > lim * lim) atomicOr(&ctl->disp_flag, 1u);
        } else {
            g_out[3 * i] = (double)g0;
            g_out[3 * i + 1] = (double)g1;
            g_out[3 * i + 2] = (double)g2;
        }
    }
    const double se = block_tree256((double)es + (double)ec, sh);
    const double sk = block_tree256((double)ks + (double)kc, sh);
    const float wm = warp_maxf(md);
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = shm[0];
        for (int w = 1; w < RCP_PAIR_THREADS / 32; ++w) bm = fmaxf(bm, shm[w]);
        part_e[blockIdx.x] = se;
        part_k[blockIdx.x] = sk;
        if (bm > 0.f) atomicMax(&ctl->maxdelta_bits, dbits((double)bm));
    }
}

// Binary64 maximum overlap over the listed pairs of the current state, same
// arithmetic as k_pair64 (confirms a binary32 stop candidate).
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
            double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            if (dx > c.halfL[0]) dx = dx - c.L[0]; else if (dx < -c.halfL[0]) dx = dx + c.L[0];
            if (dy > c.halfL[1]) dy = dy - c.L[1]; else if (dy < -c.halfL[1]) dy = dy + c.L[1];
            if (dz > c.halfL[2]) dz = dz - c.L[2]; else if (dz < -c.halfL[2]) dz = dz + c.L[2];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double dd = kappa * (0.5 * (xi.w + xj.w));
            const double delta = 1.0 - r / dd;
            if (delta > md) md = delta;
        }
    }
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_down_sync(0xffffffffu, md, o));
    if ((threadIdx.x & 31) == 0 && md > 0.0) atomicMax(&ctl->md64_bits, dbits(md));
}

// Standalone Adam step in mixed precision (rcp_adam_step): binary32 moments,
// binary64 position update, in place on the current buffer.
__global__ void k_adam_mixed(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, float* m, float* v, const double* g,
                             double eta_x)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    double4_32a* x = ctl->parity ? xB : xA;
    const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
    const float h1 = (float)(1.0 - b1), h2 = (float)(1.0 - b2);
    const float be1 = (float)c.beta1, be2 = (float)c.beta2;
    const float o1 = (float)(1.0 - c.beta1), o2 = (float)(1.0 - c.beta2);
    const float etaf = (float)eta_x, aeps = (float)c.adam_eps;
    double4_32a xi = x[i];
    double p[3] = {xi.x, xi.y, xi.z};
    for (int a = 0; a < 3; ++a) {
        const float gg = (float)g[3 * i + a];
        float mm = be1 * m[3 * i + a] + o1 * gg;
        float vv = be2 * v[3 * i + a] + o2 * (gg * gg);
        m[3 * i + a] = mm;
        v[3 * i + a] = vv;
        const float step = (etaf * (mm / h1)) / (sqrtf(vv / h2) + aeps);
        double q = p[a] - (double)step;
        if (q < 0.0) q = q + c.L[a];
        if (q >= c.L[a]) q = q - c.L[a];
        p[a] = q;
    }
    x[i] = make_double4_32a(p[0], p[1], p[2], xi.w);
}
