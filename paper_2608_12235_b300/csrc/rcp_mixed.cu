// rcp_mixed.cu -- the mixed-precision path.
//
// State of a sphere: a 32-byte record holding its position as a 56-bit fixed
// point per axis -- a 32-bit integer q_a (units of L_a 2^-32) plus a binary32
// remainder l_a in [0, 1) of those units -- and D_i^0.  That is finer than
// binary64 over most of the box (2^-56 L everywhere), and the periodic wrap is
// the wrap-around of 32-bit integer arithmetic: the minimum-image separation
// of a pair is (q_i - q_j) as a signed 32-bit integer plus (l_i - l_j),
// exactly formed to binary32 relative precision at any scale (from the largest
// spheres down to D_max / 5e5).  An axis bounded by flat walls or the
// container records [-L/2, 3L/2) instead (no wrap; spheres past a wall stay
// representable), and the wall terms take the record's position as a
// two-term binary32 sum.  Distance, overlap and the pair terms are
// binary32; each row sums them with a compensated (2Sum) accumulation; block
// and global sums are widened to binary64; the Adam moments are binary32 and
// the position update adds the step to the fixed-point record, carrying the
// integer part into q.  No binary64 operation runs per pair or per sphere in
// an iteration (binary64 throughput on B300 is a small fraction of binary32).
// Binary64 positions are derived from the records when a binary64 consumer
// needs them (neighbour build, stopping-test confirmation, shrink, export).
#include "rcp_internal.cuh"

// Axis a of a record from a binary64 coordinate: t = (x - qoff) / qspan 2^32,
// q = floor(t) (mod 2^32: a periodic x == L gives 0), l = t - q.
__device__ __forceinline__ void to_fixed(double x, const RcpConst& c, int a, int& q, float& l)
{
    double t = ((x - c.qoff[a]) / c.qspan[a]) * 4294967296.0;
    double f = floor(t);
    q = (int)(unsigned int)(unsigned long long)f;
    l = (float)(t - f);
}

__device__ __forceinline__ MixRec make_rec(double4_32a p, const RcpConst& c)
{
    MixRec r;
    to_fixed(p.x, c, 0, r.q.x, r.l.x);
    to_fixed(p.y, c, 1, r.q.y, r.l.y);
    to_fixed(p.z, c, 2, r.q.z, r.l.z);
    const float dh = (float)p.w;
    r.q.w = __float_as_int(dh);
    r.l.w = (float)(p.w - (double)dh);
    return r;
}

// D_i^0 of a record: fl32(D_i^0) and the remainder D_i^0 - fl32(D_i^0).
__device__ __forceinline__ float rec_D(const MixRec& r) { return __int_as_float(r.q.w); }
__device__ __forceinline__ float rec_Dlo(const MixRec& r) { return r.l.w; }

// Displacement a - b of two records along one axis, in length units.
__device__ __forceinline__ float rec_dx(int qa, float la, int qb, float lb, float scale)
{
    const int dq = (int)((unsigned int)qa - (unsigned int)qb);
    return ((float)dq + (la - lb)) * scale;
}

// Records from binary64 positions (positions set from outside).
__global__ void k_to_fixed(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, MixRec* rA,
                           MixRec* rB, MixRec* rb)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const int parity = ctl->parity;
    const MixRec r = make_rec((parity ? xB : xA)[i], c);
    (parity ? rB : rA)[i] = r;
    if (rb) rb[i] = r;
}

// Binary64 view of the current records, with D_i^0 from the diameter array.
__global__ void k_from_fixed(RcpCtl* ctl, RcpConst c, const MixRec* rA, const MixRec* rB, const double* D0,
                             double4_32a* xA, double4_32a* xB)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const int parity = ctl->parity;
    const MixRec r = (parity ? rB : rA)[i];
    double4_32a* x = parity ? xB : xA;
    x[i] = make_double4_32a(from_fixed(r.q.x, r.l.x, c, 0), from_fixed(r.q.y, r.l.y, c, 1),
                            from_fixed(r.q.z, r.l.z, c, 2), D0[i]);
}

// Snapshot of the current records at a neighbour build.
__global__ void k_snap_records(RcpCtl* ctl, long long N, const MixRec* rA, const MixRec* rB, MixRec* rb)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    rb[i] = (ctl->parity ? rB : rA)[i];
}

__global__ void k_mix_refresh(RcpCtl* ctl, RcpConst c) { mix_fill(ctl, c); }

// A warp's private copy of the scalars: lanes copy the stored binary32 words;
// if a source value changed since they were stored (a path that did not
// refresh them), the warp derives them itself.  Same values either way.
__device__ __forceinline__ void mix_load_warp(const RcpCtl* ctl, const RcpConst& c, MixScalars& S, int lane)
{
    const bool stale = lane < RCP_MIX_SRC && mix_src_value(ctl, lane) != ctl->mix_src[lane];
    if (__any_sync(0xffffffffu, stale)) {
        if (lane == 0) mix_scalars(ctl, c, S);
    } else if (lane < (int)(sizeof(MixScalars) / sizeof(float))) {
        reinterpret_cast<float*>(&S)[lane] = reinterpret_cast<const float*>(&ctl->mix)[lane];
    }
    __syncwarp();
}

// Adam on one axis of a record: binary32 moments, step added to the
// fixed-point position (integer part into q, fraction into l).
__device__ __forceinline__ void adam_fixed(float g, float& m, float& v, int& q, float& l, float qinv,
                                           const MixScalars& s)
{
    m = s.be1 * m + s.o1 * g;
    v = s.be2 * v + s.o2 * (g * g);
    const float step = __fdividef(s.eta * (m * s.rh1), sqrtf(v * s.rh2) + s.aeps);
    float d = -step * qinv;                      // displacement in fixed-point units
    d = fminf(fmaxf(d, -1073741824.0f), 1073741824.0f);
    const float di = floorf(d);
    const float df = d - di;                     // exact, in [0, 1)
    float ln = l + df;                           // [0, 2)
    const float carry = floorf(ln);
    ln = ln - carry;
    q = (int)((unsigned int)q + (unsigned int)(int)di + (unsigned int)(int)carry);
    l = ln;
}

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProd).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = a * b;
    e = __fmaf_rn(a, b, -p);
}

// Displacement a - b along one axis as an unevaluated binary32 sum hi + lo in
// length units, exact up to ~2^-40 relative: the integer part is split into
// its upper 24 bits and its low 8 bits (each exact in binary32, no 64-bit
// conversion) so that no digit of the remainder difference is lost.
__device__ __forceinline__ void rec_dx2(int qa, float la, int qb, float lb, float shi, float slo, float& hi,
                                        float& lo)
{
    const int dq = (int)((unsigned int)qa - (unsigned int)qb);
    const float hq = (float)((dq >> 8) * 256);   // at most 24 significant bits: exact
    const float eq = (float)(dq & 0xff);         // dq - the above, in [0, 255]: exact
    float s1, e1, x_hi, t;
    two_sum(eq, la - lb, s1, e1);
    two_sum(hq, s1, x_hi, t);
    const float x_lo = t + e1;
    float p, pe;
    two_prod(x_hi, shi, p, pe);
    hi = p;
    lo = pe + (x_hi * slo + x_lo * shi);
}

// Overlap of a pair that the binary32 pretest could not reject, with the
// cancellation in d - r removed: N = d^2 - r^2 is formed in binary32 pairs
// (d = kappa (D_i + D_j)/2 and r^2 from the split displacements), then
// u = N / d^2 and delta = 1 - sqrt(1 - u) = u / (1 + sqrt(1 - u)).  Returns
// delta (<= 0 for no overlap), r, and the displacement (binary32).
// Contact diameter of a record as an unevaluated binary32 sum: kappa D^0 for
// a mobile sphere (D^0 > 0), the fixed F = -D^0 for a frozen one (Sec. IV).
__device__ __forceinline__ void contact_diameter2(const MixRec& r, const MixScalars& S, float& hi, float& lo)
{
    const float D = rec_D(r), Dl = rec_Dlo(r);
    if (D > 0.0f) {
        float p, pe;
        two_prod(S.kappa, D, p, pe);
        hi = p;
        lo = pe + (S.kappa * Dl + S.kappa_lo * D);
    } else {
        hi = -D;
        lo = -Dl;
    }
}

// Binary32 contact diameter (the same choice).
__device__ __forceinline__ float contact_diameter(float D, const MixScalars& S) { return D > 0.0f ? S.kappa * D : -D; }

// d = kappa (D_i + D_j) / 2 of two mobile spheres as hi + lo.
__device__ __forceinline__ void mobile_pair_diameter(const MixRec& ri, const MixRec& rj, const MixScalars& S,
                                                     float& dh, float& dl)
{
    float sh, se;
    two_sum(rec_D(ri), rec_D(rj), sh, se);
    const float sl = se + (rec_Dlo(ri) + rec_Dlo(rj));
    float de;
    two_prod(S.kappa, 0.5f * sh, dh, de);
    dl = de + (S.kappa * (0.5f * sl) + S.kappa_lo * (0.5f * sh));
}

// FZ: the packing holds frozen spheres (D^0 = -F < 0), whose contact
// diameter does not scale with kappa.
template <bool FZ>
__device__ __forceinline__ float precise_delta(const MixRec& ri, const MixRec& rj, const MixScalars& S,
                                               const RcpConst& c, float& dx, float& dy, float& dz, float& r)
{
    float xh, xl, yh, yl, zh, zl;
    rec_dx2(ri.q.x, ri.l.x, rj.q.x, rj.l.x, c.qs_hi[0], c.qs_lo[0], xh, xl);
    rec_dx2(ri.q.y, ri.l.y, rj.q.y, rj.l.y, c.qs_hi[1], c.qs_lo[1], yh, yl);
    rec_dx2(ri.q.z, ri.l.z, rj.q.z, rj.l.z, c.qs_hi[2], c.qs_lo[2], zh, zl);
    // r^2
    float px, ex, py, ey, pz, ez;
    two_prod(xh, xh, px, ex);
    two_prod(yh, yh, py, ey);
    two_prod(zh, zh, pz, ez);
    float s1, t1, s2, t2;
    two_sum(px, py, s1, t1);
    two_sum(s1, pz, s2, t2);
    const float r2l = ((t1 + t2) + (ex + ey + ez)) + 2.0f * ((xh * xl + yh * yl) + zh * zl);
    // d = kappa (D_i + D_j) / 2; with a frozen sphere in the pair, the mean
    // of the two contact diameters
    float dh, dl;
    if constexpr (FZ) {
        if (rec_D(ri) > 0.0f && rec_D(rj) > 0.0f) {
            mobile_pair_diameter(ri, rj, S, dh, dl);
        } else {
            float ai, ei, aj, ej, sh, se;
            contact_diameter2(ri, S, ai, ei);
            contact_diameter2(rj, S, aj, ej);
            two_sum(ai, aj, sh, se);
            dh = 0.5f * sh;
            dl = 0.5f * (se + (ei + ej));
        }
    } else {
        mobile_pair_diameter(ri, rj, S, dh, dl);
    }
    // d^2 - r^2
    float d2h, d2e;
    two_prod(dh, dh, d2h, d2e);
    const float d2l = d2e + 2.0f * dh * dl;
    float nh, ne;
    two_sum(d2h, -s2, nh, ne);
    const float n = nh + (ne + (d2l - r2l));
    dx = xh;
    dy = yh;
    dz = zh;
    r = sqrtf(s2);
    if (!(n > 0.0f)) return n;
    const float u = __fdividef(n, d2h);
    return __fdividef(u, 1.0f + sqrtf(1.0f - u));
}

// Binary32 pre-test on the integer parts of two records (the first 16 bytes):
// false when the pair certainly does not overlap.  Leaving out the
// remainders moves each axis by less than one fixed-point unit, the whole
// displacement by less than sqrt(3) units, so the pair is kept whenever
// r_q <= d (1 + 1e-5) + 2 units (c.qmargin), r_q the distance of the integer
// parts; the binary32 roundings of r_q^2 and d (a few 2^-24 each) sit far
// inside the 1e-5.
template <bool FZ>
__device__ __forceinline__ bool pretest_q(const int4& qi, const int4& qj, const MixScalars& S, const RcpConst& c)
{
    const float fx = (float)(int)((unsigned int)qi.x - (unsigned int)qj.x) * c.qscale[0];
    const float fy = (float)(int)((unsigned int)qi.y - (unsigned int)qj.y) * c.qscale[1];
    const float fz = (float)(int)((unsigned int)qi.z - (unsigned int)qj.z) * c.qscale[2];
    const float r2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, fz * fz));
    float d;
    if constexpr (FZ)
        d = 0.5f * (contact_diameter(__int_as_float(qi.w), S) + contact_diameter(__int_as_float(qj.w), S));
    else
        d = S.kappa * (0.5f * (__int_as_float(qi.w) + __int_as_float(qj.w)));
    const float T = __fmaf_rn(d, 1.00001f, c.qmargin);
    return !(r2 > T * T);
}

__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ int4 load_q(const MixRec* r, unsigned int j)
{
    return __ldg(reinterpret_cast<const int4*>(r) + 2 * (size_t)j);
}

// Gradient term of a pair that passed the pre-test (zero when the precise
// overlap is not positive or the centres coincide, and for a frozen row);
// the j > i share of e and k goes into (es, ec), (ks, kc), the overlap into
// md.  With a frozen sphere in the pair, d d / d kappa is half the mobile
// D^0 rather than d / kappa, so k takes eps delta (1 - delta) (mobile parts)
// / (2 d).
template <bool FZ>
__device__ __forceinline__ void pair_term_precise(const MixRec& ri, const MixRec& rj, long long i, unsigned int j,
                                                  const MixScalars& S, const RcpConst& c, float& t0, float& t1,
                                                  float& t2, float& es, float& ec, float& ks, float& kc, float& md)
{
    float dx, dy, dz, r;
    t0 = t1 = t2 = 0.0f;
    const float delta = precise_delta<FZ>(ri, rj, S, c, dx, dy, dz, r);
    if (!(delta > 0.0f)) return;
    float dd;
    bool mob = true, grad_row = true;
    if constexpr (FZ) {
        const float Di = rec_D(ri), Dj = rec_D(rj);
        mob = Di > 0.0f && Dj > 0.0f;
        grad_row = Di > 0.0f;
        dd = mob ? S.kappa * (0.5f * (Di + Dj)) : 0.5f * (contact_diameter(Di, S) + contact_diameter(Dj, S));
    } else {
        dd = S.kappa * (0.5f * (rec_D(ri) + rec_D(rj)));
    }
    if (r > 0.0f && grad_row) {
        const float coef = __fdividef(S.eps * delta, dd * r);
        t0 = -coef * dx;
        t1 = -coef * dy;
        t2 = -coef * dz;
    }
    if ((long long)j > i) {
        acc2(es, ec, (0.5f * S.eps) * (delta * delta));
        if constexpr (FZ) {
            const float ek = (S.eps * delta) * (1.0f - delta);
            acc2(ks, kc, mob ? ek * S.rkappa
                             : __fdividef(ek * (0.5f * (fmaxf(rec_D(ri), 0.0f) + fmaxf(rec_D(rj), 0.0f))), dd));
        } else {
            acc2(ks, kc, ((S.eps * delta) * (1.0f - delta)) * S.rkappa);
        }
    }
    md = fmaxf(md, delta);
}

// Skin budget of a record against its build snapshot (binary32 with 1e-5
// margins): what its displacement leaves for kappa growth,
// b_i = 2 (theta sigma_i - |x_i - x_i^b|) / D_i; negative flags the rebuild.
__device__ __forceinline__ float skin_budget32(RcpCtl* ctl, const RcpConst& c, const MixScalars& S, const MixRec& rn,
                                               const MixRec& b)
{
    const float ex = rec_dx(rn.q.x, rn.l.x, b.q.x, b.l.x, c.qscale[0]);
    const float ey = rec_dx(rn.q.y, rn.l.y, b.q.y, b.l.y, c.qscale[1]);
    const float ez = rec_dx(rn.q.z, rn.l.z, b.q.z, b.l.z, c.qscale[2]);
    const float disp = sqrtf(__fmaf_rn(ex, ex, __fmaf_rn(ey, ey, ez * ez))) * 1.00001f;
    const float sig = __fmaf_rn(S.limA, rec_D(rn), S.limB);
    const float bi = 2.0f * (sig - disp) / rec_D(rn) * 0.99999f;
    if (!(bi >= 0.0f)) {
        atomicOr(&ctl->disp_flag, 1u);
        return INFINITY;
    }
    return bi;
}

__device__ __forceinline__ void push_budget32(RcpCtl* ctl, float bud)
{
    for (int o = 16; o > 0; o >>= 1) bud = fminf(bud, __shfl_down_sync(0xffffffffu, bud, o));
    if ((threadIdx.x & 31) == 0 && bud < INFINITY) {
        const unsigned int bits = __float_as_uint(bud);
        if (bits < *(volatile unsigned int*)&ctl->kbud_bits) atomicMin(&ctl->kbud_bits, bits);
    }
}

// Close row i: the Adam step of its record (Adam mode) or its gradient out.
// Returns the row's skin budget (infinity in gradient mode).
template <bool FZ>
__device__ __forceinline__ float row_epilogue(RcpCtl* ctl, const RcpConst& c, const MixScalars& S, long long i,
                                              const MixRec& ri, float g0, float g1, float g2, float* m, float* v,
                                              MixRec* rout, const MixRec* rb, int mode, double* g_out)
{
    if constexpr (FZ) {
        if (!(rec_D(ri) > 0.0f)) {
            // a frozen sphere: no Adam step (its record carries over to the
            // other buffer), no gradient, no skin use
            if (mode == RCP_MODE_ADAM) {
                rout[i] = ri;
            } else {
                g_out[3 * i] = 0.0;
                g_out[3 * i + 1] = 0.0;
                g_out[3 * i + 2] = 0.0;
            }
            return INFINITY;
        }
    }
    if (mode == RCP_MODE_ADAM) {
        MixRec rn = ri;
        float m0 = m[3 * i], m1 = m[3 * i + 1], m2 = m[3 * i + 2];
        float v0 = v[3 * i], v1 = v[3 * i + 1], v2 = v[3 * i + 2];
        adam_fixed(g0, m0, v0, rn.q.x, rn.l.x, c.qinv[0], S);
        adam_fixed(g1, m1, v1, rn.q.y, rn.l.y, c.qinv[1], S);
        adam_fixed(g2, m2, v2, rn.q.z, rn.l.z, c.qinv[2], S);
        m[3 * i] = m0; m[3 * i + 1] = m1; m[3 * i + 2] = m2;
        v[3 * i] = v0; v[3 * i + 1] = v1; v[3 * i + 2] = v2;
        rout[i] = rn;
        return skin_budget32(ctl, c, S, rn, rb[i]);
    }
    g_out[3 * i] = (double)g0;
    g_out[3 * i + 1] = (double)g1;
    g_out[3 * i + 2] = (double)g2;
    return INFINITY;
}

__device__ __forceinline__ float warp_sum(float s)
{
    for (int o = 16; o > 0; o >>= 1) s = s + __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}


// Coordinate of a record along axis a as an unevaluated binary32 sum
// (length units): qoff + (q + l) qspan 2^-32, the integer part split into its
// upper 24 and low 8 bits (each exact), so exact to ~2^-44 of the span.
__device__ __forceinline__ void rec_pos2(int qv, float l, const RcpConst& c, int a, float& hi, float& lo)
{
    const unsigned int q = (unsigned int)qv;
    const float hq = (float)(q & 0xffffff00u), eq = (float)(q & 0xffu);
    float s1, e1, xh, t;
    two_sum(eq, l, s1, e1);
    two_sum(hq, s1, xh, t);
    const float xl = t + e1;
    float p, pe;
    two_prod(xh, c.qs_hi[a], p, pe);
    const float l1 = pe + (xh * c.qs_lo[a] + xl * c.qs_hi[a]);
    float s2, e2;
    two_sum(p, c.qo_hi[a], s2, e2);
    hi = s2;
    lo = e2 + (l1 + c.qo_lo[a]);
}

// One wall contact of a sphere of radius rad = rh + rl at clearance h = hh +
// hl: delta = (rad - h) / rad with the difference taken in two-term
// arithmetic (no cancellation near contact); energy eps/2 delta^2, and for a
// mobile sphere the force eps delta / rad (returned) and the kappa term eps
// delta (1 - delta) / kappa, 1 - delta taken as h / rad (d delta / d kappa =
// (h / rad) / kappa; no cancellation where the centre sits on the wall and
// delta is near 1).  Returns false when the sphere clears the wall.
template <bool FZ>
__device__ __forceinline__ bool wall_contact(float hh, float hl, float rh, float rl, bool mob, const MixScalars& S,
                                             float& es, float& ec, float& ks, float& kc, float& md, float& f)
{
    float nh, ne;
    two_sum(rh, -hh, nh, ne);
    const float n = nh + (ne + (rl - hl));
    if (!(n > 0.0f)) return false;
    const float delta = __fdividef(n, rh);
    acc2(es, ec, (0.5f * S.eps) * (delta * delta));
    f = 0.0f;
    if (!FZ || mob) {
        f = __fdividef(S.eps * delta, rh);
        acc2(ks, kc, ((S.eps * delta) * __fdividef(hh + hl, rh)) * S.rkappa);
    }
    md = fmaxf(md, delta);
    return true;
}

// A row's wall terms after its pairs (Sec. II boundaries): the flat walls at
// 0 and L_a of every walled axis (h = x_a, then h = L_a - x_a), then the
// curved container, h = R - |x - centre| over its axes (d h / d x_a =
// -(x_a - c_a) / |x - c|).  Positions, clearances and distances in two-term
// binary32, so a contact within 1e-8 of the radius still resolves.  A frozen
// row takes the energy and the overlap but no force and no kappa term.
// A pre-test on the integer parts alone skips the two-term work of a sphere
// that clears every wall: x_a ~ fl32(q_a) qscale_a + qoff_a is within a few
// 2^-24 L_a of the coordinate (the conversion of q_a keeps 24 bits, the
// remainder is below one unit), so a clearance above rad + 2^-20 L_a
// (c.wmargin) is certain.
template <bool FZ>
__device__ __forceinline__ void wall_terms32(const RcpConst& c, const MixScalars& S, const MixRec& ri, float& g0,
                                             float& c0, float& g1, float& c1, float& g2, float& c2, float& es,
                                             float& ec, float& ks, float& kc, float& md)
{
    bool mob = true;
    if constexpr (FZ) mob = rec_D(ri) > 0.0f;
    float rh, rl;
    contact_diameter2(ri, S, rh, rl);
    rh *= 0.5f;
    rl *= 0.5f;
    const int qa[3] = {ri.q.x, ri.q.y, ri.q.z};
    const float la[3] = {ri.l.x, ri.l.y, ri.l.z};
    float xc[3];
    for (int a = 0; a < 3; ++a)
        xc[a] = __fmaf_rn(__uint2float_rn((unsigned int)qa[a]), c.qscale[a], c.qo_hi[a]);
    for (int a = 0; a < 3; ++a) {
        if (!((c.walls >> a) & 1)) continue;
        if (fminf(xc[a], c.Lf[a] - xc[a]) > rh + c.wmargin) continue;   // clears both walls of the axis
        float xh, xl;
        rec_pos2(qa[a], la[a], c, a, xh, xl);
        float& g = a == 0 ? g0 : (a == 1 ? g1 : g2);
        float& gc = a == 0 ? c0 : (a == 1 ? c1 : c2);
        float f;
        if (wall_contact<FZ>(xh, xl, rh, rl, mob, S, es, ec, ks, kc, md, f) && f != 0.0f) acc2(g, gc, -f);
        float s, e;
        two_sum(c.Lf[a], -xh, s, e);
        if (wall_contact<FZ>(s, e + (c.Llo[a] - xl), rh, rl, mob, S, es, ec, ks, kc, md, f) && f != 0.0f)
            acc2(g, gc, f);
    }
    if (c.container) {
        float q2 = 0.0f;
        for (int a = 0; a < 3; ++a)
            if ((c.caxes >> a) & 1) {
                const float o = xc[a] - 0.5f * c.Lf[a];
                q2 = __fmaf_rn(o, o, q2);
            }
        const float clear = c.Rc_hi - rh - c.wmargin;   // certainly inside the ball / cylinder
        if (clear > 0.0f && q2 < clear * clear * (1.0f - 1e-5f)) return;
        float oh[3] = {0.f, 0.f, 0.f};
        float d2h = 0.0f, d2l = 0.0f;
        for (int a = 0; a < 3; ++a) {
            if (!((c.caxes >> a) & 1)) continue;
            float xh, xl;
            rec_pos2(qa[a], la[a], c, a, xh, xl);
            // offset from the centre L_a / 2 (exact halves of Lf and Llo)
            float s, e;
            two_sum(xh, -0.5f * c.Lf[a], s, e);
            const float ol = e + (xl - 0.5f * c.Llo[a]);
            float oh2, ol2;
            two_sum(s, ol, oh2, ol2);
            oh[a] = oh2;
            float p, pe;
            two_prod(oh2, oh2, p, pe);
            float t, te;
            two_sum(d2h, p, t, te);
            d2h = t;
            d2l = d2l + (te + (pe + 2.0f * oh2 * ol2));
        }
        // |x - c| = sqrt(d2) as hi + lo (one Newton correction)
        const float dh = sqrtf(d2h);
        const float dl = dh > 0.0f ? __fdividef(__fmaf_rn(-dh, dh, d2h) + d2l, 2.0f * dh) : 0.0f;
        // h = R - |x - c|
        float s, e;
        two_sum(c.Rc_hi, -dh, s, e);
        float f;
        if (wall_contact<FZ>(s, e + (c.Rc_lo - dl), rh, rl, mob, S, es, ec, ks, kc, md, f) && f != 0.0f && dh > 0.0f) {
            const float fr = __fdividef(f, dh);
            if (c.caxes & 1) acc2(g0, c0, fr * oh[0]);
            if (c.caxes & 2) acc2(g1, c1, fr * oh[1]);
            if (c.caxes & 4) acc2(g2, c2, fr * oh[2]);
        }
    }
}

// The pair kernel of the mixed path.  Listed entries far outnumber
// overlapping pairs (about 3 % in the dense packings at S = 5e5, where most
// small spheres rattle in the voids of the large ones), so every row is taken
// in two passes: pass 1 puts each listed partner through pretest_q, which
// reads only the first 16 bytes of its record, and keeps a bit per partner
// that may overlap; pass 2 takes the marked partners, in the row's order,
// through the precise terms (so the sums are those of a single walk).
// Blocks [0, c.long_blocks) give one warp to each row longer than c.long_row
// (the rows of the largest spheres, holding hundreds of small neighbours):
// lanes stride over the row, four strides per round trip to memory, and the
// gradient is reduced with compensated shuffles.  The other blocks give one
// thread to each remaining row, four partners per round trip; the row's
// moments, build snapshot and own record are requested into L2 as the row
// starts, so the Adam epilogue does not wait on DRAM.  The kernel is bound by
// the latency of the col -> record chains, not by DRAM bytes or L1 traffic.
// Both parts end with the row's Adam step (or its gradient out); block
// partials of e and k go to part_e/part_k.  The order of every sum depends only on the
// list, so results are reproducible run to run.
#ifndef RCP_MIX_MINB
#define RCP_MIX_MINB 5   // resident blocks per SM the register budget is sized for (48 registers)
#endif
__device__ __forceinline__ void prefetch_row(const float* m, const float* v, const MixRec* rb, const MixRec* rin,
                                             long long i)
{
    prefetch_l2(m + 3 * i);
    prefetch_l2(v + 3 * i);
    prefetch_l2(rb + i);
    prefetch_l2(rin + i);
}
#define RCP_MIX_WARPS (RCP_PAIR_THREADS / 32)

__device__ __forceinline__ unsigned int lanemask_lt(int lane) { return (1u << lane) - 1u; }

// WL: the packing has flat walls or a container (wall terms per row).
template <bool FZ, bool WL>
__device__ __forceinline__ void pair_mixed_body(RcpCtl* ctl, const RcpConst& c, float* m, float* v, MixRec* rA,
                                                MixRec* rB, const unsigned int* rowptr, const unsigned int* col,
                                                const unsigned int* long_rows, const MixRec* rb, double* part_e, double* part_k, int mode,
                                                double* g_out, unsigned int blk)
{
    const unsigned int FULL = 0xffffffffu;
    __shared__ MixScalars Sw[RCP_MIX_WARPS];
    if (ctl->halted) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    MixScalars& S = Sw[warp];
    mix_load_warp(ctl, c, S, lane);
    const int parity = ctl->parity;
    const MixRec* __restrict__ rin = parity ? rB : rA;
    MixRec* __restrict__ rout = parity ? rA : rB;
    float es = 0.f, ec = 0.f, ks = 0.f, kc = 0.f, md = 0.f;
    float bud = INFINITY;
    if (blk < c.long_blocks) {
        const unsigned int nlong = ctl->n_long;
        const unsigned int nw = c.long_blocks * RCP_MIX_WARPS;
        for (unsigned int r = blk * RCP_MIX_WARPS + warp; r < nlong; r += nw) {
            const long long i = long_rows[r];
            const int4 qi = load_q(rin, (unsigned int)i);
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
            const unsigned int t1 = rowptr[i + 1];
            // windows of 32 warp strides: pass 1 marks, per lane, the strides
            // whose partner may overlap (four strides per round trip to
            // memory); pass 2 takes those in order through the precise terms
            for (unsigned int w0 = rowptr[i] + lane; w0 < t1; w0 += 32u * 32u) {
                unsigned int hit = 0u;
                unsigned int m = 0u;
                for (; m < 32u && w0 + 32u * (m + 3u) < t1; m += 4u) {
                    const unsigned int t = w0 + 32u * m;
                    const unsigned int j0 = col[t], j1 = col[t + 32], j2 = col[t + 64], j3 = col[t + 96];
                    const int4 q0 = load_q(rin, j0), q1 = load_q(rin, j1), q2 = load_q(rin, j2), q3 = load_q(rin, j3);
                    if (pretest_q<FZ>(qi, q0, S, c)) hit |= 1u << m;
                    if (pretest_q<FZ>(qi, q1, S, c)) hit |= 2u << m;
                    if (pretest_q<FZ>(qi, q2, S, c)) hit |= 4u << m;
                    if (pretest_q<FZ>(qi, q3, S, c)) hit |= 8u << m;
                }
                for (; m < 32u && w0 + 32u * m < t1; ++m)
                    if (pretest_q<FZ>(qi, load_q(rin, col[w0 + 32u * m]), S, c)) hit |= 1u << m;
                if (hit) {
                    const MixRec ri = rin[i];
                    do {
                        const unsigned int k = (unsigned int)__ffs(hit) - 1u;
                        hit &= hit - 1u;
                        const unsigned int j = col[w0 + 32u * k];
                        float a0, a1, a2;
                        pair_term_precise<FZ>(ri, rin[j], i, j, S, c, a0, a1, a2, es, ec, ks, kc, md);
                        acc2(g0, c0, a0);
                        acc2(g1, c1, a1);
                        acc2(g2, c2, a2);
                    } while (hit);
                }
            }
            // lanes' compensated sums, then a plain tree over the lanes: each
            // lane's s + c is its terms' sum to ~2^-24, the tree adds five
            // roundings of the lane sums' magnitude
            g0 = warp_sum(g0 + c0);
            g1 = warp_sum(g1 + c1);
            g2 = warp_sum(g2 + c2);
            if (lane == 0) {
                if constexpr (WL) {
                    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
                    wall_terms32<FZ>(c, S, rin[i], g0, e0, g1, e1, g2, e2, es, ec, ks, kc, md);
                    g0 += e0;
                    g1 += e1;
                    g2 += e2;
                }
                bud = fminf(bud, row_epilogue<FZ>(ctl, c, S, i, rin[i], g0, g1, g2, m, v, rout, rb, mode, g_out));
            }
        }
    } else {
        // one thread per row
        const long long i = (long long)(blk - c.long_blocks) * RCP_PAIR_THREADS + threadIdx.x;
        if (i < c.N) {
            const unsigned int t0 = rowptr[i], t1 = rowptr[i + 1];
            if (t1 - t0 <= c.long_row) {
                // the epilogue's streams, requested now so that they wait in
                // L2 rather than on the row's last round trip
                if (mode == RCP_MODE_ADAM) prefetch_row(m, v, rb, rin, i);
                const int4 qi = load_q(rin, (unsigned int)i);
                // pass 1: the pre-test marks the partners that may overlap (a
                // row holds at most 32 entries here, four per round trip to
                // memory)
                unsigned int hit = 0u;
                unsigned int t = t0;
                for (; t + 4 <= t1; t += 4) {
                    const unsigned int j0 = col[t], j1 = col[t + 1], j2 = col[t + 2], j3 = col[t + 3];
                    const int4 q0 = load_q(rin, j0), q1 = load_q(rin, j1), q2 = load_q(rin, j2), q3 = load_q(rin, j3);
                    if (pretest_q<FZ>(qi, q0, S, c)) hit |= 1u << (t - t0);
                    if (pretest_q<FZ>(qi, q1, S, c)) hit |= 2u << (t - t0);
                    if (pretest_q<FZ>(qi, q2, S, c)) hit |= 4u << (t - t0);
                    if (pretest_q<FZ>(qi, q3, S, c)) hit |= 8u << (t - t0);
                }
                for (; t + 2 <= t1; t += 2) {
                    const unsigned int j0 = col[t], j1 = col[t + 1];
                    const int4 q0 = load_q(rin, j0), q1 = load_q(rin, j1);
                    if (pretest_q<FZ>(qi, q0, S, c)) hit |= 1u << (t - t0);
                    if (pretest_q<FZ>(qi, q1, S, c)) hit |= 2u << (t - t0);
                }
                if (t < t1 && pretest_q<FZ>(qi, load_q(rin, col[t]), S, c)) hit |= 1u << (t - t0);
                // pass 2: the marked partners through the precise terms, in
                // the row's order
                const MixRec ri = rin[i];
                float g0 = 0.f, g1 = 0.f, g2 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
                while (hit) {
                    const unsigned int k = (unsigned int)__ffs(hit) - 1u;
                    hit &= hit - 1u;
                    const unsigned int j = col[t0 + k];
                    float a0, a1, a2;
                    pair_term_precise<FZ>(ri, rin[j], i, j, S, c, a0, a1, a2, es, ec, ks, kc, md);
                    acc2(g0, c0, a0);
                    acc2(g1, c1, a1);
                    acc2(g2, c2, a2);
                }
                if constexpr (WL) wall_terms32<FZ>(c, S, ri, g0, c0, g1, c1, g2, c2, es, ec, ks, kc, md);
                bud = row_epilogue<FZ>(ctl, c, S, i, ri, g0 + c0, g1 + c1, g2 + c2, m, v, rout, rb, mode, g_out);
            }
        }
    }
    push_budget32(ctl, bud);
    // most lanes hold no overlap: lane 0 adds the others' compensated sums
    // in lane order (the same order whatever the timing)
    unsigned int nz = __ballot_sync(FULL, es != 0.f || ec != 0.f || ks != 0.f || kc != 0.f) & ~1u;
    while (nz) {
        const int l = __ffs(nz) - 1;
        nz &= nz - 1u;
        const float se = __shfl_sync(FULL, es, l), sec = __shfl_sync(FULL, ec, l);
        const float sk = __shfl_sync(FULL, ks, l), skc = __shfl_sync(FULL, kc, l);
        if (lane == 0) {
            acc2(es, ec, se);
            ec = ec + sec;
            acc2(ks, kc, sk);
            kc = kc + skc;
        }
    }
    const float wm = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(md)));   // md >= 0
    // the block's partials: warp 0 adds the warps' compensated sums in warp
    // order (a block retires only when its last warp ends, so the barrier
    // holds no resource longer), one (sum, correction) pair per block
    __shared__ float4 s_part[RCP_MIX_WARPS];
    __shared__ float s_max[RCP_MIX_WARPS];
    if (lane == 0) {
        s_part[warp] = make_float4(es, ec, ks, kc);
        s_max[warp] = wm;
    }
    __syncthreads();
    if (warp == 0) {
        const float4 p = lane < RCP_MIX_WARPS ? s_part[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float bm = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(lane < RCP_MIX_WARPS ? s_max[lane] : 0.f)));
        if (lane == 0) {
            float be = p.x, bec = p.y, bk = p.z, bkc = p.w;
            for (int w = 1; w < RCP_MIX_WARPS; ++w) {
                const float4 q = s_part[w];
                acc2(be, bec, q.x);
                bec = bec + q.y;
                acc2(bk, bkc, q.z);
                bkc = bkc + q.w;
            }
            reinterpret_cast<float2*>(part_e)[blk] = make_float2(be, bec);
            reinterpret_cast<float2*>(part_k)[blk] = make_float2(bk, bkc);
            if (bm > 0.f) {
                const unsigned long long b = dbits((double)bm);
                if (b > *(volatile unsigned long long*)&ctl->maxdelta_bits) atomicMax(&ctl->maxdelta_bits, b);
            }
        }
    }
}

__global__ void __launch_bounds__(RCP_PAIR_THREADS, RCP_MIX_MINB)
k_pair_mixed(RcpCtl* ctl, RcpConst c, float* m, float* v, MixRec* rA, MixRec* rB, const unsigned int* rowptr,
             const unsigned int* col, const unsigned int* long_rows, const MixRec* rb, double* part_e,
             double* part_k, int mode, double* g_out)
{
    pair_mixed_body<false, false>(ctl, c, m, v, rA, rB, rowptr, col, long_rows, rb, part_e, part_k, mode, g_out,
                                  blockIdx.x);
}

// The same for a packing that holds frozen spheres (seated stages of the
// cascade, Sec. IV).
__global__ void __launch_bounds__(RCP_PAIR_THREADS, RCP_MIX_MINB)
k_pair_mixed_fz(RcpCtl* ctl, RcpConst c, float* m, float* v, MixRec* rA, MixRec* rB, const unsigned int* rowptr,
                const unsigned int* col, const unsigned int* long_rows, const MixRec* rb, double* part_e,
                double* part_k, int mode, double* g_out)
{
    pair_mixed_body<true, false>(ctl, c, m, v, rA, rB, rowptr, col, long_rows, rb, part_e, part_k, mode, g_out,
                                 blockIdx.x);
}

// The same for a packing bounded by flat walls or a container (Sec. II),
// frozen spheres or not.
__global__ void __launch_bounds__(RCP_PAIR_THREADS, RCP_MIX_MINB)
k_pair_mixed_wl(RcpCtl* ctl, RcpConst c, float* m, float* v, MixRec* rA, MixRec* rB, const unsigned int* rowptr,
                const unsigned int* col, const unsigned int* long_rows, const MixRec* rb, double* part_e,
                double* part_k, int mode, double* g_out)
{
    pair_mixed_body<true, true>(ctl, c, m, v, rA, rB, rowptr, col, long_rows, rb, part_e, part_k, mode, g_out,
                                blockIdx.x);
}

__device__ __forceinline__ int batch_pack_m(const unsigned int* bstart, int B, unsigned int block)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bstart[mid] <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched mixed pair kernel: block b serves packing p with local block
// b - bstart[p], so each packing computes exactly what its own launch would.
// FZ: some packing of the batch holds frozen spheres; WL: walls or a container.
template <bool FZ, bool WL>
__device__ __forceinline__ void pair_mixed_batch_body(const PackDev* P, const unsigned int* bstart, int B, int mode)
{
    const int p = batch_pack_m(bstart, B, blockIdx.x);
    const PackDev& q = P[p];
    pair_mixed_body<FZ, WL>(q.ctl, q.c, q.m32, q.v32, q.rA, q.rB, q.rowptr, q.col, q.long_rows, q.rb, q.part_e,
                        q.part_k, mode, q.g, blockIdx.x - bstart[p]);
}

__global__ void __launch_bounds__(RCP_PAIR_THREADS, RCP_MIX_MINB)
k_pair_mixed_batch(const PackDev* P, const unsigned int* bstart, int B, int mode)
{
    pair_mixed_batch_body<false, false>(P, bstart, B, mode);
}

__global__ void __launch_bounds__(RCP_PAIR_THREADS, RCP_MIX_MINB)
k_pair_mixed_batch_fz(const PackDev* P, const unsigned int* bstart, int B, int mode)
{
    pair_mixed_batch_body<true, false>(P, bstart, B, mode);
}

__global__ void __launch_bounds__(RCP_PAIR_THREADS, RCP_MIX_MINB)
k_pair_mixed_batch_wl(const PackDev* P, const unsigned int* bstart, int B, int mode)
{
    pair_mixed_batch_body<true, true>(P, bstart, B, mode);
}

// Standalone Adam step in mixed precision (rcp_adam_step): binary32 moments
// on the fixed-point records, in place, with the skin check.
__global__ void k_adam_mixed(RcpCtl* ctl, RcpConst c, MixRec* rA, MixRec* rB, float* m, float* v, const double* g,
                             const MixRec* rb, double eta_x)
{
    __shared__ MixScalars S;
    if (threadIdx.x == 0) {
        mix_scalars(ctl, c, S);
        S.eta = (float)eta_x;
    }
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float bud = INFINITY;
    if (i < c.N) {
        MixRec* r = ctl->parity ? rB : rA;
        MixRec rn = r[i];
        if (rec_D(rn) > 0.0f) {   // a frozen sphere does not move
            for (int a = 0; a < 3; ++a) {
                float mm = m[3 * i + a], vv = v[3 * i + a];
                int* q = a == 0 ? &rn.q.x : (a == 1 ? &rn.q.y : &rn.q.z);
                float* l = a == 0 ? &rn.l.x : (a == 1 ? &rn.l.y : &rn.l.z);
                adam_fixed((float)g[3 * i + a], mm, vv, *q, *l, c.qinv[a], S);
                m[3 * i + a] = mm;
                v[3 * i + a] = vv;
            }
            r[i] = rn;
            bud = skin_budget32(ctl, c, S, rn, rb[i]);
        }
    }
    push_budget32(ctl, bud);
}
