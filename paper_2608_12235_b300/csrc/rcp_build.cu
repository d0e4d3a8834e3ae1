// rcp_build.cu -- the size-stratified multilevel cell grid and the Verlet
// list (the B300 replacement of the k-d tree of App. A).
//
// Every sphere gets an interaction radius rho_i = kappa_b D_i^0 (1/2 + s) +
// sigma0 (half its diameter plus its skin); a pair is listed iff its
// minimum-image distance is below rho_i + rho_j.  Spheres are binned into
// size classes by rho (class k holds rho in (rho_max 2^-(k+1), rho_max
// 2^-k]), each class with its own uniform grid of power-of-two cells per
// axis, sized by occupancy (a cell holds about `cell_occupancy` spheres of
// its class; any cell size is correct because the search scans every cell
// within its radius).  Particles are ordered by the key (class, cz, cy, cx)
// with a counting sort over the dense per-class cell table (counts, a scan,
// a scatter, each cell's spheres sorted by index), and the table holds each
// cell's range [start, end) in that order.  A sphere scans its
// own class and every finer class over the cells within its search radius;
// a pair inside one class is found from both ends, a pair across classes
// from the coarser end only, which emits both directions.  The pairs (row << b
// | col) become CSR rows with ascending columns (per-row counts, a scatter
// into the rows, a shared-memory sort of each row).  Integer and
// exact-predicate work only: the list is bit-identical to the definition.
#include "rcp_internal.cuh"

__device__ __forceinline__ double min_image_b(double t, double L, double h)
{
    if (t > h) t = t - L;
    else if (t < -h) t = t + L;
    return t;
}

__global__ void k_build_begin(RcpCtl* ctl, double sigma0)
{
    ctl->kappa_b = ctl->kappa;
    ctl->sigma0 = sigma0;
    ctl->rho_max_bits = 0ull;
    for (int k = 0; k < RCP_KMAX; ++k) {
        ctl->rho_lvl_bits[k] = 0ull;
        ctl->lvl_count[k] = 0ull;
        ctl->rho_lvl[k] = 0.0;
    }
    ctl->nlev = 0;
    ctl->pair_cursor = 0ull;
}

// Interaction radii, their maximum, and a binary32 copy of every sphere for
// the search's prefilter: (x/L_x, y/L_y, z/L_z, rho) rounded to binary32.
__global__ void __launch_bounds__(256) k_rho(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                                             double* rho, float4* xf)
{
    __shared__ double sh[8];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (i < c.N) {
        const double4_32a p = (ctl->parity ? xB : xA)[i];
        r = size_at(p.w, ctl->kappa_b) * (0.5 + c.skin_s) + ctl->sigma0;   // frozen: fixed diameter
        rho[i] = r;
        xf[i] = make_float4((float)(p.x * c.invL[0]), (float)(p.y * c.invL[1]), (float)(p.z * c.invL[2]), (float)r);
    }
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) r = fmax(r, sh[w]);
        if (r > 0.0) atomicMax(&ctl->rho_max_bits, dbits(r));
    }
}

// Mixed path: the same radii and binary32 copy from the fixed-point records,
// with no binary64 view of the positions.  On a periodic axis u_a =
// fl32(q_a) 2^-32 drops the remainder (below one unit, 2^-32) and rounds q_a
// to 24 bits, so it is within 2^-25 + 2^-32 of x_a / L_a -- the prefilter's
// error budget for fl32(x_a / L_a) (2^-25) grows by under 1 %, far inside
// its margins.  A bounded axis (its record spans [-L/2, 3L/2)) takes
// fl32(x_a / L_a) of the binary64 coordinate, as k_rho does.  rho_i from
// D_i^0 exactly as k_rho forms it.
__device__ __forceinline__ float unit_coord(const int4& qr, const float4& lr, const RcpConst& c, int a)
{
    const int q = a == 0 ? qr.x : (a == 1 ? qr.y : qr.z);
    if ((c.bounded >> a) & 1) {
        const float l = a == 0 ? lr.x : (a == 1 ? lr.y : lr.z);
        return (float)(from_fixed(q, l, c, a) * c.invL[a]);
    }
    return __uint2float_rn((unsigned int)q) * 0x1.0p-32f;
}

__global__ void __launch_bounds__(256) k_rho_mixed(RcpCtl* ctl, RcpConst c, const MixRec* rA, const MixRec* rB,
                                                   const double* D0, double* rho, float4* xf)
{
    __shared__ double sh[8];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (i < c.N) {
        // the integer parts alone unless an axis is bounded (half the bytes)
        const MixRec* R = ctl->parity ? rB : rA;
        const int4 q = reinterpret_cast<const int4*>(R)[2 * i];
        const float4 l = c.bounded ? reinterpret_cast<const float4*>(R)[2 * i + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        r = size_at(D0[i], ctl->kappa_b) * (0.5 + c.skin_s) + ctl->sigma0;
        rho[i] = r;
        xf[i] = make_float4(unit_coord(q, l, c, 0), unit_coord(q, l, c, 1), unit_coord(q, l, c, 2), (float)r);
    }
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) r = fmax(r, sh[w]);
        if (r > 0.0) atomicMax(&ctl->rho_max_bits, dbits(r));
    }
}

// Mixed path: the per-sphere state in cell-key order (sphere t of the new
// order is sphere sorted[t] of the old), so that the rows a warp evaluates
// lie in neighbouring cells of one size class and their partners sit close
// together in memory.  Records and the binary64 view of the current parity go
// to the other buffers (k_flip_parity then makes them current); moments,
// diameters, radii, classes and the caller-order map go to the scratch arrays.
__global__ void k_permute_state(const RcpCtl* ctl, long long N, const unsigned int* sorted, MixRec* rA, MixRec* rB,
                                double4_32a* xA, double4_32a* xB, const float* m, const float* v, float* m2,
                                float* v2, const double* D0, double* D02, const double* rho, double* rho2,
                                const int* lvl, int* lvl2, const unsigned int* perm, unsigned int* perm2)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int parity = ctl->parity;
    const long long s = sorted[t];
    (parity ? rA : rB)[t] = (parity ? rB : rA)[s];
    if (xA) (parity ? xA : xB)[t] = (parity ? xB : xA)[s];   // binary64 view, when the build uses one
    for (int a = 0; a < 3; ++a) {
        m2[3 * t + a] = m[3 * s + a];
        v2[3 * t + a] = v[3 * s + a];
    }
    D02[t] = D0[s];
    rho2[t] = rho[s];
    lvl2[t] = lvl[s];
    perm2[t] = perm[s];
}

__global__ void k_flip_parity(RcpCtl* ctl) { ctl->parity ^= 1; }

__global__ void k_iota(long long N, unsigned int* out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) out[t] = (unsigned int)t;
}

// The binary32 copies in cell order, so the candidates of one cell are
// contiguous.
__global__ void k_gather_sorted(long long N, const unsigned int* idx_sorted, const float4* xf, float4* xsf)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) xsf[t] = xf[idx_sorted[t]];
}

// Class k_i = max{k in [0, 31] : rho_i 2^k <= rho_max} (exact power-of-two
// scaling), the largest rho and the size of each class (aggregated per block
// in shared memory, then one atomic per class and block).
__global__ void __launch_bounds__(256) k_level(RcpCtl* ctl, long long N, const double* rho, int* lvl)
{
    __shared__ unsigned long long smax[RCP_KMAX];
    __shared__ unsigned int scnt[RCP_KMAX];
    if (threadIdx.x < RCP_KMAX) {
        smax[threadIdx.x] = 0ull;
        scnt[threadIdx.x] = 0u;
    }
    __syncthreads();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const unsigned long long bm = ctl->rho_max_bits;
        const double r = rho[i];
        const unsigned long long br = dbits(r);
        const int er = (int)(br >> 52), em = (int)(bm >> 52);   // biased exponents (r, rho_max > 0)
        int k;
        if (er > 0) {
            // r 2^k <= rho_max  <=>  (er + k, fraction of r) <= (em, fraction of rho_max)
            const unsigned long long fmask = (1ull << 52) - 1ull;
            k = em - er - ((br & fmask) > (bm & fmask) ? 1 : 0);
            k = k < 0 ? 0 : (k > RCP_KMAX - 1 ? RCP_KMAX - 1 : k);
        } else {
            // subnormal radius: the plain search over k
            const double rmax = bitsd(bm);
            k = 0;
            while (k + 1 < RCP_KMAX && ldexp(r, k + 1) <= rmax) ++k;
        }
        lvl[i] = k;
        atomicMax(&smax[k], dbits(r));
        atomicAdd(&scnt[k], 1u);
    }
    __syncthreads();
    if (threadIdx.x < RCP_KMAX && scnt[threadIdx.x]) {
        atomicMax(&ctl->rho_lvl_bits[threadIdx.x], smax[threadIdx.x]);
        atomicAdd(&ctl->lvl_count[threadIdx.x], (unsigned long long)scnt[threadIdx.x]);
    }
}

// Cells per axis of each class: the largest power of two n <= 2^19 whose
// cell holds at least c.cell_occ spheres of the class on average
// (h^3 count >= cell_occ V, h = L/n).  The search scans every cell within
// its radius, so any cell size is correct; this one balances cell-table lookups
// against candidates.  Also the periodic-image rule: every listed pair must
// be closer than half a box edge, i.e. 4 rho_max < min L.
__global__ void k_grid(RcpCtl* ctl, RcpConst c)
{
    // one thread per (class, axis)
    const int t = threadIdx.x;
    if (t < RCP_KMAX * 3) {
        const int k = t / 3, a = t % 3;
        const double r = bitsd(ctl->rho_lvl_bits[k]);
        const double cnt = (double)ctl->lvl_count[k];
        if (a == 0) {
            ctl->rho_lvl[k] = r;
            ctl->rho_lvl_f[k] = (float)r;
        }
        unsigned int n = 1;
        if (r > 0.0 && a < c.dim)   // d = 2: one cell layer in z, area occupancy in x and y
            for (;;) {
                if (n >= RCP_NMAX_AXIS) break;
                const double h = c.L[a] / (double)(2 * n);
                const double cell = c.dim == 2 ? h * h : (h * h) * h;
                if (!(cell * cnt >= c.cell_occ * c.V)) break;
                n *= 2;
            }
        ctl->ng[k][a] = (int)n;
    }
    __syncthreads();
    if (t != 0) return;
    int nlev = 0;
    for (int k = 0; k < RCP_KMAX; ++k)
        if (ctl->rho_lvl[k] > 0.0) nlev = k + 1;
    ctl->nlev = nlev;
    unsigned long long off = 0;
    for (int k = 0; k <= RCP_KMAX; ++k) {
        ctl->cell_off[k] = off;
        if (k < nlev && ctl->rho_lvl[k] > 0.0)
            off += (unsigned long long)ctl->ng[k][0] * (unsigned long long)ctl->ng[k][1] *
                   (unsigned long long)ctl->ng[k][2];
    }
    const double rmax = bitsd(ctl->rho_max_bits);
    if (!(4.0 * rmax < c.Lmin)) {
        ctl->status = RCP_ERR_IMAGE;
        ctl->halted = 1;
    }
}

// fl(x / L) n, floored: with L a power of two the quotient is the product
// with 1 / L, exactly (both are the correctly rounded x 2^-e), which spares a
// binary64 division per axis.
__device__ __forceinline__ unsigned int cell_of(double x, double L, double invL, bool pow2, unsigned int n)
{
    double f = floor((pow2 ? x * invL : x / L) * (double)n);
    long long cc = (long long)f;
    if (cc < 0) cc = 0;
    if (cc > (long long)n - 1) cc = (long long)n - 1;
    return (unsigned int)cc;
}

__device__ __forceinline__ unsigned long long pack_key(unsigned int k, unsigned int cz, unsigned int cy,
                                                       unsigned int cx)
{
    return ((unsigned long long)k << 57) | ((unsigned long long)cz << 38) | ((unsigned long long)cy << 19) |
           (unsigned long long)cx;
}

__global__ void k_cell_key(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const int* lvl,
                           unsigned long long* key)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double4_32a* x = ctl->parity ? xB : xA;
    const double4_32a p = x[i];
    const int k = lvl[i];
    unsigned int cx = cell_of(p.x, c.L[0], c.invL[0], c.pow2L & 1, (unsigned int)ctl->ng[k][0]);
    unsigned int cy = cell_of(p.y, c.L[1], c.invL[1], c.pow2L & 2, (unsigned int)ctl->ng[k][1]);
    unsigned int cz = cell_of(p.z, c.L[2], c.invL[2], c.pow2L & 4, (unsigned int)ctl->ng[k][2]);
    key[i] = pack_key((unsigned int)k, cz, cy, cx);
}

// Mixed path: the cell of a record from its integer part alone.  With n = 2^b
// cells per axis, floor((q + l) 2^-32 n) = q >> (32 - b) because l < 1: the
// same cell as floor(fl(x/L) n) for the binary64 position the record was made
// from (q = floor(fl(x/L) 2^32)), in integer arithmetic.  On a bounded axis
// the record spans [-L/2, 3L/2): x/L = (q + l) 2^-31 - 1/2, so the cell is
// (q >> (31 - b)) - n/2, clamped to the grid as cell_of clamps it (a sphere
// past a wall stays in the edge cell; the search's windows carry margins
// wider than the rounding at a cell edge).
__device__ __forceinline__ unsigned int cell_q(int q, unsigned int n, bool bounded)
{
    if (n <= 1u) return 0u;
    const int b = 31 - __clz(n);
    if (!bounded) return (unsigned int)q >> (32 - b);
    int v = (int)((unsigned int)q >> (31 - b)) - (int)(n >> 1);
    v = v < 0 ? 0 : (v > (int)n - 1 ? (int)n - 1 : v);
    return (unsigned int)v;
}

__global__ void k_cell_key_mixed(RcpCtl* ctl, RcpConst c, const MixRec* rA, const MixRec* rB, const int* lvl,
                                 unsigned long long* key)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const int4 q = reinterpret_cast<const int4*>(ctl->parity ? rB : rA)[2 * i];
    const int k = lvl[i];
    key[i] = pack_key((unsigned int)k, cell_q(q.z, (unsigned int)ctl->ng[k][2], (c.bounded >> 2) & 1),
                      cell_q(q.y, (unsigned int)ctl->ng[k][1], (c.bounded >> 1) & 1),
                      cell_q(q.x, (unsigned int)ctl->ng[k][0], c.bounded & 1));
}

// Exclusive scan, 4096 items per block (1024 threads x 4); block totals are
// written out and scanned recursively by the host, then added back.
__global__ void __launch_bounds__(1024)
k_scan_block(const unsigned int* in, long long n, unsigned int* out, unsigned int* totals)
{
    __shared__ unsigned int ws[32];
    const long long base = (long long)blockIdx.x * 4096 + (long long)threadIdx.x * 4;
    unsigned int a[4], s = 0;
    for (int q = 0; q < 4; ++q) {
        a[q] = (base + q < n) ? in[base + q] : 0u;
        s += a[q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned int w = ws[lane];
        unsigned int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        ws[lane] = wi - w;  // exclusive prefix of the warp totals
        if (lane == 31 && totals) totals[blockIdx.x] = wi;
    }
    __syncthreads();
    unsigned int run = ws[warp] + incl - s;
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) out[base + q] = run;
        run += a[q];
    }
}

__global__ void k_scan_add(unsigned int* out, long long n, const unsigned int* offs)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] += offs[t / 4096];
}

// ---------------------------------------------------------------------------
// Dense cell table: for every cell of every size class, the range [x, y) of
// its spheres in the sorted order (empty cells stay (0, 0)).  A class with
// count spheres has at most count / cell_occupancy cells (k_grid), so the
// table holds at most N / cell_occupancy entries; class k starts at
// ctl->cell_off[k] and is laid out (z, y, x) row-major.
__device__ __forceinline__ unsigned long long cell_index(const RcpCtl* ctl, unsigned int k, unsigned int cz,
                                                         unsigned int cy, unsigned int cx)
{
    return ctl->cell_off[k] +
           ((unsigned long long)cz * (unsigned int)ctl->ng[k][1] + cy) * (unsigned int)ctl->ng[k][0] + cx;
}

// Spheres sorted by cell: a counting sort through the CSR kernels, with the
// cells as rows.  k_cell_pairs forms (cell index << nbits | sphere); the
// cell index orders the cells as the key (class, cz, cy, cx) does, so the
// rows, each sorted by sphere index (k_row_sort), give exactly the order a
// stable sort of the cell keys gives.
__global__ void k_cell_pairs(const RcpCtl* ctl, long long N, const unsigned long long* key, int nbits,
                             unsigned long long* ck)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned long long k = key[i];
    const unsigned long long m = (1ull << 19) - 1ull;
    const unsigned long long ci = cell_index(ctl, (unsigned int)(k >> 57), (unsigned int)((k >> 38) & m),
                                             (unsigned int)((k >> 19) & m), (unsigned int)(k & m));
    ck[i] = (ci << nbits) | (unsigned long long)i;
}

// The dense cell table from the cells' row pointers: [start, end) per cell.
__global__ void k_cell_table(const unsigned int* cptr, unsigned long long ncells, uint2* cells)
{
    const unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncells) cells[c] = make_uint2(cptr[c], cptr[c + 1]);
}

// The sorted keys (key position t holds the key of sphere sorted[t]).
__global__ void k_gather_keys(long long N, const unsigned int* sorted, const unsigned long long* key,
                              unsigned long long* skeys)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) skeys[t] = key[sorted[t]];
}

// ---------------------------------------------------------------------------
// Pair search, one pass.  Threads take the spheres in cell-key order.  Each
// thread keeps the entries it finds in a small local buffer; a full buffer is
// flushed to the global array through one atomic reservation, and the final
// flush is aggregated over the warp.  The order of entries in the array is
// arbitrary (the CSR pass orders them); entries beyond `cap` are counted but
// not written, and the host re-runs the search with a larger array.  The
// inclusion test is the exact binary64 predicate
// dx^2 + dy^2 + dz^2 < (rho_i + rho_j)^2  (minimum image).
#define RCP_SEARCH_BUF 32
// a window of at least this many cells goes to k_search_heavy, in chunks of
// RCP_SEARCH_CHUNK cells, one warp each
#ifndef RCP_SEARCH_HEAVY
#define RCP_SEARCH_HEAVY 32
#endif
#define RCP_SEARCH_CHUNK 64

// Minimum-image component in box units (d = u_i - u_j in (-1, 1)): d minus
// its nearest integer, exact (d - 1 for d in [1/2, 1) is exact by Sterbenz's
// lemma), and +-1/2 stay as they are (round half to even gives 0 there).
__device__ __forceinline__ float wrap_unit(float d) { return d - rintf(d); }

// The class-k cells within reach of a sphere at ui (box units, radius ui.w):
// per axis the first cell (before the periodic wrap), the count and the grid.
struct SearchWin {
    int lo[3];
    unsigned int nc[3], ng[3];
};

__device__ __forceinline__ SearchWin search_window(const RcpCtl* ctl, const RcpConst& c, const float4& ui, int k)
{
    SearchWin w;
    const float rk = ctl->rho_lvl_f[k];
    const float u3[3] = {ui.x, ui.y, ui.z};
    for (int a = 0; a < 3; ++a) {
        w.ng[a] = (unsigned int)ctl->ng[k][a];
        // search radius in box units, in binary32: rho_i, rho_k and 1/L_a are
        // each within 2^-24 of their binary64 values and the sum and product
        // round twice more, a few 1e-7 in all, far inside the 1e-6 relative
        // margin; 2e-6 covers the rounding of u (a window only has to be wide
        // enough)
        const float Ru = __fmaf_rn((ui.w + rk) * c.invLf[a], 1.000001f, 2e-6f);
        const float fn = (float)w.ng[a];
        int l = (int)floorf((u3[a] - Ru) * fn);
        int h = (int)floorf((u3[a] + Ru) * fn);
        if ((c.bounded >> a) & 1) {
            // bounded axis, no wrap: clamp the window (the edge cells also
            // hold the spheres beyond the walls)
            const int top = (int)w.ng[a] - 1;
            l = l < 0 ? 0 : (l > top ? top : l);
            h = h < 0 ? 0 : (h > top ? top : h);
            w.lo[a] = l;
            w.nc[a] = (unsigned int)(h - l + 1);
        } else if (h - l + 1 >= (int)w.ng[a]) {
            w.lo[a] = 0;
            w.nc[a] = w.ng[a];
        } else {
            w.lo[a] = l;
            w.nc[a] = (unsigned int)(h - l + 1);
        }
    }
    return w;
}

// Range [start, end) of the window's cell (cx, cy, cz) in the class-k table.
__device__ __forceinline__ uint2 window_cell(const uint2* ck, const SearchWin& w, unsigned int cx, unsigned int cy,
                                             unsigned int cz)
{
    const unsigned int z = (unsigned int)(w.lo[2] + (int)cz) & (w.ng[2] - 1);
    const unsigned int y = (unsigned int)(w.lo[1] + (int)cy) & (w.ng[1] - 1);
    const unsigned int x = (unsigned int)(w.lo[0] + (int)cx) & (w.ng[0] - 1);
    return ck[((unsigned long long)z * w.ng[1] + y) * w.ng[0] + x];
}

// Binary32 prefilter with rigorous bounds.  With u = fl32(x/L) (error <=
// 2^-25 per coordinate) the binary32 distance r_f of a pair satisfies
// |r_f - r| <= 1e-6 r + 5e-7 Lmax (the rounding analysis gives 2.3e-7 r +
// 1.6e-7 Lmax), and fl32(rho_i) + fl32(rho_j) is within 1.2e-7 of rho_i +
// rho_j (relative).  The accept and reject thresholds carry 2e-6 relative
// margins on top; pairs inside the band where those bounds cannot decide are
// settled by the exact binary64 predicate, so the listed set is exactly the
// binary64 one.
__device__ __forceinline__ double4_32a rec_position(const MixRec& r, const RcpConst& c)
{
    return make_double4_32a(from_fixed(r.q.x, r.l.x, c, 0), from_fixed(r.q.y, r.l.y, c, 1),
                            from_fixed(r.q.z, r.l.z, c, 2), 0.0);
}

// Candidate t (a sorted position) against sphere i: its index j when the
// pair is listed (j != i), else 0xffffffff.  The band's binary64 positions
// come from the records when the build has no binary64 view (recs != NULL),
// the values the view would hold.
__device__ __forceinline__ unsigned int listed_partner(const RcpConst& c, float Eabs, const double4_32a* x,
                                                       const MixRec* recs, const double* rho,
                                                       const unsigned int* idx_sorted, const float4* xsf,
                                                       unsigned int t, long long i, const float4& ui, double ri)
{
    const float up = 1.0f + 2e-6f, dn = 1.0f - 2e-6f;
    const float4 uj = xsf[t];
    const float dx = ((c.bounded & 1) ? ui.x - uj.x : wrap_unit(ui.x - uj.x)) * c.Lf[0];
    const float dy = ((c.bounded & 2) ? ui.y - uj.y : wrap_unit(ui.y - uj.y)) * c.Lf[1];
    const float dz = ((c.bounded & 4) ? ui.z - uj.z : wrap_unit(ui.z - uj.z)) * c.Lf[2];
    const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
    const float cut = ui.w + uj.w;
    const float hi = (cut * up + Eabs) * up;
    if (r2 > hi * hi) return 0xffffffffu;            // certainly not listed
    const unsigned int j = idx_sorted ? idx_sorted[t] : t;
    if ((long long)j == i) return 0xffffffffu;
    const float lo_in = (cut * dn - Eabs) * dn;
    if (lo_in > 0.0f && r2 < lo_in * lo_in) return j;  // certainly listed
    // the band: exact binary64 predicate
    const double4_32a xi = recs ? rec_position(recs[i], c) : x[i];
    const double4_32a xj = recs ? rec_position(recs[j], c) : x[j];
    const double ex = (c.bounded & 1) ? xi.x - xj.x : min_image_b(xi.x - xj.x, c.L[0], c.halfL[0]);
    const double ey = (c.bounded & 2) ? xi.y - xj.y : min_image_b(xi.y - xj.y, c.L[1], c.halfL[1]);
    const double ez = (c.bounded & 4) ? xi.z - xj.z : min_image_b(xi.z - xj.z, c.L[2], c.halfL[2]);
    const double d2 = ex * ex + ey * ey + ez * ez;
    const double cc = ri + rho[j];
    return d2 < cc * cc ? j : 0xffffffffu;
}

template <class F>
__device__ __forceinline__ void scan_cell(const RcpConst& c, float Eabs, const double4_32a* x, const MixRec* recs,
                                          const double* rho, const unsigned int* idx_sorted, const float4* xsf,
                                          uint2 range, long long i, const float4& ui, double ri, F&& hit)
{
    for (unsigned int t = range.x; t < range.y; ++t) {
        const unsigned int j = listed_partner(c, Eabs, x, recs, rho, idx_sorted, xsf, t, i, ui, ri);
        if (j != 0xffffffffu) hit(j);
    }
}

// A thread's buffer of list entries (row << nbits | col).
struct EntryBuf {
    unsigned long long b[RCP_SEARCH_BUF];
    int n;

    __device__ __forceinline__ void flush_to(unsigned long long* pairs, unsigned long long cap,
                                             unsigned long long base) const
    {
        for (int q = 0; q < n; ++q)
            if (base + q < cap) pairs[base + q] = b[q];
    }
    // the entry (i, j), and (j, i) too when `both`
    __device__ __forceinline__ void put(RcpCtl* ctl, unsigned long long* pairs, unsigned long long cap, int nbits,
                                        unsigned long long i, unsigned long long j, bool both)
    {
        if (n + (both ? 2 : 1) > RCP_SEARCH_BUF) {
            flush_to(pairs, cap, atomicAdd(&ctl->pair_cursor, (unsigned long long)n));
            n = 0;
        }
        b[n++] = (i << nbits) | j;
        if (both) b[n++] = (j << nbits) | i;
    }
    // warp-aggregated final flush (every lane of the warp calls it)
    __device__ __forceinline__ void flush_warp(RcpCtl* ctl, unsigned long long* pairs, unsigned long long cap)
    {
        const int lane = threadIdx.x & 31;
        unsigned int incl = (unsigned int)n;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && total) base = atomicAdd(&ctl->pair_cursor, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 31);
        flush_to(pairs, cap, base + (incl - (unsigned int)n));
        n = 0;
    }
};

// The first lane whose inclusive count exceeds v (31 when none does).
__device__ __forceinline__ int warp_owner(unsigned int incl, unsigned int v)
{
    int o = 0;
    for (int b = 16; b > 0; b >>= 1)
        if (__shfl_sync(0xffffffffu, incl, o + b - 1) <= v) o += b;
    return o;
}

__device__ __forceinline__ unsigned int warp_incl_scan(unsigned int v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Queue a window of ncell cells for k_search_heavy: one item (sphere,
// chunk << 5 | class) per chunk of RCP_SEARCH_CHUNK cells.  False when the
// queue is full (its slots are then marked empty and the caller scans the
// window itself).
__device__ __forceinline__ bool queue_window(RcpCtl* ctl, uint2* heavy, unsigned int heavy_cap, long long ts, int k,
                                             unsigned long long ncell)
{
    if (ncell >= (1ull << 31)) return false;
    const unsigned int nch = (unsigned int)((ncell + RCP_SEARCH_CHUNK - 1) / RCP_SEARCH_CHUNK);
    const unsigned int s = atomicAdd(&ctl->search_heavy, nch);
    if ((unsigned long long)s + nch <= heavy_cap) {
        for (unsigned int h = 0; h < nch; ++h) heavy[s + h] = make_uint2((unsigned int)ts, (h << 5) | (unsigned int)k);
        return true;
    }
    for (unsigned long long h = s; h < heavy_cap && h < (unsigned long long)s + nch; ++h)
        heavy[h] = make_uint2(0xffffffffu, 0u);
    return false;
}

// The list search.  Sphere i of class l_i scans its own class and every
// finer one (k >= l_i): a pair inside one class is found from both ends, a
// pair across classes from the coarser end only, which emits both
// directions.  Searching from the coarse end keeps the windows' cell slack
// small: a window over the fine grid exceeds 2 (rho_i + rho_k) by one fine
// cell per axis, whereas a fine sphere's window over a coarse grid exceeds it
// by a coarse cell, which then holds many candidates that are out of reach.
// A window of RCP_SEARCH_HEAVY cells or more (the largest spheres over the
// finest grid) is queued for k_search_heavy, which gives it a warp.  The
// other windows of a warp's 32 spheres (one class at a time) are laid end
// to end, first cell by cell and then candidate by candidate, and the lanes
// take them 32 at a time: each lane tests one candidate for whichever sphere
// owns it, so the lanes stay busy however the windows and cells differ
// (when each lane walked its own sphere's window, 9 of 32 lanes were busy).
// Threads take the spheres in cell-key order (size class, then cell), so a
// warp shares its size class and most of its cells; idx_sorted is NULL when
// the state itself is in that order.
// (64 registers, 4 blocks per SM: the unbounded build took 76 and ran 1.5x
// slower for the lost occupancy)
__global__ void __launch_bounds__(256, 4)
k_search(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const MixRec* rA, const MixRec* rB,
         const double* rho, const int* lvl, const unsigned int* idx_sorted, const float4* xsf, const uint2* cells,
         unsigned long long* pairs, unsigned long long cap, int nbits, uint2* heavy, unsigned int heavy_cap)
{
    const unsigned int FULL = 0xffffffffu;
    const MixRec* recs = rA ? (ctl->parity ? rB : rA) : nullptr;
    const long long ts = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool act = ts < c.N;
    const float Eabs = (float)(5e-7 * c.Lmax);
    const double4_32a* x = ctl->parity ? xB : xA;
    long long i = 0;
    float4 ui = make_float4(0.f, 0.f, 0.f, 0.f);
    double ri = 0.0;
    int li = RCP_KMAX;
    if (act) {
        i = idx_sorted ? (long long)idx_sorted[ts] : ts;
        ui = xsf[ts];
        ri = rho[i];
        li = lvl[i];
    }
    EntryBuf eb;
    eb.n = 0;
    const int nlev = ctl->nlev;
    for (int k = 0; k < nlev; ++k) {   // warp-uniform
        SearchWin w = {{0, 0, 0}, {0u, 0u, 0u}, {1u, 1u, 1u}};
        unsigned int ncell = 0u;   // this lane's light window
        if (k >= li && ctl->rho_lvl_f[k] > 0.0f) {
            w = search_window(ctl, c, ui, k);
            const unsigned long long nc = (unsigned long long)w.nc[0] * w.nc[1] * w.nc[2];
            if (nc < RCP_SEARCH_HEAVY) {
                ncell = (unsigned int)nc;
            } else if (!queue_window(ctl, heavy, heavy_cap, ts, k, nc)) {
                // queue full: this lane walks the window by itself
                const bool both = k > li;
                const uint2* ck = cells + ctl->cell_off[k];
                for (unsigned int cz = 0; cz < w.nc[2]; ++cz)
                    for (unsigned int cy = 0; cy < w.nc[1]; ++cy)
                        for (unsigned int cx = 0; cx < w.nc[0]; ++cx)
                            scan_cell(c, Eabs, x, recs, rho, idx_sorted, xsf, window_cell(ck, w, cx, cy, cz), i, ui,
                                      ri, [&](unsigned int j) { eb.put(ctl, pairs, cap, nbits, i, j, both); });
            }
        }
        const unsigned int cin = warp_incl_scan(ncell, lane);
        const unsigned int C = __shfl_sync(FULL, cin, 31);   // < 32 RCP_SEARCH_HEAVY
        if (C == 0u) continue;
        const uint2* ck = cells + ctl->cell_off[k];
        const unsigned int ng0 = (unsigned int)ctl->ng[k][0], ng1 = (unsigned int)ctl->ng[k][1];
        const unsigned int ng2 = (unsigned int)ctl->ng[k][2];
        for (unsigned int cb = 0; cb < C; cb += 32u) {   // warp-uniform rounds of 32 cells
            const unsigned int cc = cb + (unsigned int)lane;
            const int o = warp_owner(cin, cc);   // the lane whose window holds cell cc
            const unsigned int e = cc - (__shfl_sync(FULL, cin, o) - __shfl_sync(FULL, ncell, o));
            const int lo0 = __shfl_sync(FULL, w.lo[0], o), lo1 = __shfl_sync(FULL, w.lo[1], o);
            const int lo2 = __shfl_sync(FULL, w.lo[2], o);
            const unsigned int n0 = __shfl_sync(FULL, w.nc[0], o), n1 = __shfl_sync(FULL, w.nc[1], o);
            uint2 range = make_uint2(0u, 0u);
            if (cc < C) {
                const unsigned int n01 = n0 * n1;
                const unsigned int cz = e / n01, r = e - cz * n01;
                const unsigned int cy = r / n0, cx = r - cy * n0;
                const unsigned int zz = (unsigned int)(lo2 + (int)cz) & (ng2 - 1u);
                const unsigned int yy = (unsigned int)(lo1 + (int)cy) & (ng1 - 1u);
                const unsigned int xx = (unsigned int)(lo0 + (int)cx) & (ng0 - 1u);
                range = ck[((unsigned long long)zz * ng1 + yy) * ng0 + xx];
            }
            const unsigned int cnt = range.y - range.x;
            const unsigned int tin = warp_incl_scan(cnt, lane);
            const unsigned int T = __shfl_sync(FULL, tin, 31);
            for (unsigned int tb = 0; tb < T; tb += 32u) {   // warp-uniform rounds of 32 candidates
                const unsigned int tt = tb + (unsigned int)lane;
                const int L = warp_owner(tin, tt);   // the lane holding that candidate's cell
                const unsigned int cand =
                    __shfl_sync(FULL, range.x, L) + (tt - (__shfl_sync(FULL, tin, L) - __shfl_sync(FULL, cnt, L)));
                const int so = __shfl_sync(FULL, o, L);   // the lane of the sphere that owns the cell
                const float4 us = make_float4(__shfl_sync(FULL, ui.x, so), __shfl_sync(FULL, ui.y, so),
                                              __shfl_sync(FULL, ui.z, so), __shfl_sync(FULL, ui.w, so));
                const double rs = __shfl_sync(FULL, ri, so);
                const long long is = __shfl_sync(FULL, i, so);
                const int ls = __shfl_sync(FULL, li, so);
                if (tt < T) {
                    const unsigned int j = listed_partner(c, Eabs, x, recs, rho, idx_sorted, xsf, cand, is, us, rs);
                    if (j != 0xffffffffu) eb.put(ctl, pairs, cap, nbits, is, j, k > ls);
                }
                // buffers past half full go out with one reservation per warp
                if (__any_sync(FULL, eb.n > RCP_SEARCH_BUF / 2)) eb.flush_warp(ctl, pairs, cap);
            }
        }
    }
    eb.flush_warp(ctl, pairs, cap);
}

// The queued chunks of windows, one warp each.  Each round the lanes read
// the ranges of 32 cells, a warp scan of their counts lays the candidates end
// to end, and the lanes take the candidates 32 at a time (the owning cell by a
// binary search over the scan), so the lanes stay busy whatever the cells
// hold.  The grid strides over the queue, whose length the device holds.
__global__ void __launch_bounds__(256)
k_search_heavy(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const MixRec* rA,
               const MixRec* rB, const double* rho, const int* lvl, const unsigned int* idx_sorted,
               const float4* xsf, const uint2* cells, unsigned long long* pairs, unsigned long long cap, int nbits,
               const uint2* heavy, unsigned int heavy_cap)
{
    const MixRec* recs = rA ? (ctl->parity ? rB : rA) : nullptr;
    const unsigned int FULL = 0xffffffffu;
    const unsigned int lane = threadIdx.x & 31;
    const unsigned int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned int nw = (gridDim.x * blockDim.x) >> 5;
    const unsigned int nq = min(ctl->search_heavy, heavy_cap);
    const double4_32a* x = ctl->parity ? xB : xA;
    const float Eabs = (float)(5e-7 * c.Lmax);
    EntryBuf eb;
    eb.n = 0;
    for (unsigned int q = w0; q < nq; q += nw) {   // warp-uniform
        const uint2 item = heavy[q];
        if (item.x == 0xffffffffu) continue;        // a slot of a window scanned in place
        const long long ts = item.x;
        const int k = (int)(item.y & 31u);
        const long long i = idx_sorted ? (long long)idx_sorted[ts] : ts;
        const float4 ui = xsf[ts];
        const double ri = rho[i];
        const bool both = k > lvl[i];
        const SearchWin w = search_window(ctl, c, ui, k);
        const uint2* ck = cells + ctl->cell_off[k];
        const unsigned int nxy = w.nc[0] * w.nc[1], ncell = nxy * w.nc[2];
        const unsigned int e_lo = (item.y >> 5) * RCP_SEARCH_CHUNK;
        const unsigned int e_hi = min(ncell, e_lo + RCP_SEARCH_CHUNK);
        for (unsigned int e0 = e_lo; e0 < e_hi; e0 += 32) {   // warp-uniform rounds of 32 cells
            const unsigned int e = e0 + lane;
            uint2 range = make_uint2(0u, 0u);
            if (e < e_hi) {
                const unsigned int cz = e / nxy, r = e - cz * nxy;
                const unsigned int cy = r / w.nc[0], cx = r - cy * w.nc[0];
                range = window_cell(ck, w, cx, cy, cz);
            }
            const unsigned int cnt = range.y - range.x;
            unsigned int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(FULL, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const unsigned int total = __shfl_sync(FULL, incl, 31);
            for (unsigned int cb = 0; cb < total; cb += 32) {   // warp-uniform
                const unsigned int cc = cb + lane;
                // owner: the first lane whose inclusive count exceeds cc
                int o = 0;
                for (int b = 16; b > 0; b >>= 1)
                    if (__shfl_sync(FULL, incl, o + b - 1) <= cc) o += b;
                const unsigned int first = __shfl_sync(FULL, range.x, o);
                const unsigned int before = __shfl_sync(FULL, incl - cnt, o);
                if (cc < total) {
                    const unsigned int j =
                        listed_partner(c, Eabs, x, recs, rho, idx_sorted, xsf, first + (cc - before), i, ui, ri);
                    if (j != 0xffffffffu) eb.put(ctl, pairs, cap, nbits, i, j, both);
                }
                if (__any_sync(FULL, eb.n > RCP_SEARCH_BUF / 2)) eb.flush_warp(ctl, pairs, cap);
            }
        }
    }
    eb.flush_warp(ctl, pairs, cap);
}

// Placement rounds: the candidates of class kcur (those not yet placed) scan
// their own class and every coarser one (and, with frozen spheres, every
// class: frozen spheres of finer classes are placed before any class is); an
// overlapping pair marks the candidate that must give way.
__global__ void __launch_bounds__(256)
k_place_conflicts(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const double* rho,
                  const int* lvl, const unsigned int* idx_sorted, const float4* xsf, const uint2* cells,
                  const double* D0, const unsigned char* placed, unsigned char* reject, int kcur)
{
    const long long ts = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ts >= c.N) return;
    const long long i = idx_sorted ? (long long)idx_sorted[ts] : ts;
    // every overlap with a placed sphere or a class-mate is found from the
    // candidate's side
    if (placed[i] || lvl[i] != kcur) return;
    const double4_32a* x = ctl->parity ? xB : xA;
    const float4 ui = xsf[ts];
    const double ri = rho[i];
    const int li = lvl[i];
    const int kend = c.nfrozen > 0 ? ctl->nlev - 1 : li;
    const float Eabs = (float)(5e-7 * c.Lmax);
    if (c.walls | c.container) {   // a candidate must keep off the walls too (distance below rho_i)
        const double4_32a xi = x[i];
        for (int a = 0; a < 3; ++a) {
            if (!((c.walls >> a) & 1)) continue;
            const double xa = a == 0 ? xi.x : (a == 1 ? xi.y : xi.z);
            if (xa < ri || c.L[a] - xa < ri) reject[i] = 1;
        }
        if (c.container) {   // distance to the curved wall R - |x - c| over its axes
            double s2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                if (!((c.caxes >> a) & 1)) continue;
                const double o = (a == 0 ? xi.x : (a == 1 ? xi.y : xi.z)) - c.halfL[a];
                s2 = s2 + o * o;
            }
            if (c.Rc - sqrt(s2) < ri) reject[i] = 1;
        }
    }
    for (int k = 0; k <= kend; ++k) {
        if (!(ctl->rho_lvl_f[k] > 0.0f)) continue;
        const SearchWin w = search_window(ctl, c, ui, k);
        const uint2* ck = cells + ctl->cell_off[k];
        for (unsigned int cz = 0; cz < w.nc[2]; ++cz)
            for (unsigned int cy = 0; cy < w.nc[1]; ++cy)
                for (unsigned int cx = 0; cx < w.nc[0]; ++cx)
                    scan_cell(c, Eabs, x, nullptr, rho, idx_sorted, xsf, window_cell(ck, w, cx, cy, cz), i, ui, ri,
                              [&](unsigned int j) {
                                  // i gives way to a placed sphere and to a
                                  // class-mate candidate that precedes it
                                  // (larger D0, then lower index); spheres of
                                  // later classes are not there yet
                                  if (placed[j]) reject[i] = 1;
                                  else if (lvl[j] == kcur) {
                                      const bool j_first = D0[j] > D0[i] || (D0[j] == D0[i] && (long long)j < i);
                                      reject[j_first ? i : (long long)j] = 1;
                                  }
                              });
    }
}

// ---------------------------------------------------------------------------
// CSR rows from the unsorted pair keys (row << nbits | col) without a global
// sort: k_row_count counts the entries of every row, an exclusive scan of the
// counts is rowptr, k_row_scatter drops every column into its row's segment
// (an atomic cursor per row: arbitrary order inside the segment), and
// k_row_sort sorts each segment in shared memory.  Columns within a row are
// distinct, so the sorted list is unique: the same rows and columns, in the
// same order, as a full sort of the keys, whatever the order of the atomics.
// Within a warp, lanes of the same row share one atomic (__match_any_sync).
__global__ void k_row_count(const unsigned long long* pairs, long long P, int nbits, unsigned int* cnt)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned int r = t < P ? (unsigned int)(pairs[t] >> nbits) : 0xffffffffu;
    const unsigned int peers = __match_any_sync(0xffffffffu, r);
    if (t < P && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[r], (unsigned int)__popc(peers));
}

__global__ void k_row_scatter(const unsigned long long* pairs, long long P, int nbits, const unsigned int* rowptr,
                              unsigned int* fill, unsigned int* colu)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long key = t < P ? pairs[t] : ~0ull;
    const unsigned int r = t < P ? (unsigned int)(key >> nbits) : 0xffffffffu;
    const unsigned int peers = __match_any_sync(0xffffffffu, r);
    const int lane = threadIdx.x & 31, lead = __ffs(peers) - 1;
    unsigned int base = 0;
    if (t < P && lane == lead) base = atomicAdd(&fill[r], (unsigned int)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (t < P) colu[rowptr[r] + base + __popc(peers & ((1u << lane) - 1u))] = (unsigned int)(key & ((1ull << nbits) - 1ull));
}

// Sort of the segment [a, a + len) of v ascending: insertion sort by one
// thread (short rows).
__device__ __forceinline__ void sort_serial(unsigned int* v, unsigned int len)
{
    for (unsigned int q = 1; q < len; ++q) {
        const unsigned int x = v[q];
        unsigned int p = q;
        while (p > 0 && v[p - 1] > x) {
            v[p] = v[p - 1];
            --p;
        }
        v[p] = x;
    }
}

// Bitonic sort of v[0, len) by one warp (rows longer than 32), in the form
// whose comparators all put the smaller value first: each merge of blocks of
// k starts by comparing element i with its mirror i ^ (k - 1), then halves.
// The network runs over the next power of two with the missing elements as
// +infinity, which then never move, so a comparator that reaches past len is
// skipped.
__device__ __forceinline__ void sort_warp(unsigned int* v, unsigned int len, int lane)
{
    unsigned int n2 = 1;
    while (n2 < len) n2 <<= 1;
    for (unsigned int k = 2; k <= n2; k <<= 1) {
        for (unsigned int j = k >> 1; j > 0; j >>= 1) {
            for (unsigned int i = (unsigned int)lane; i < n2; i += 32) {
                const unsigned int l = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
                if (l > i && l < len) {
                    const unsigned int a = v[i], b = v[l];
                    if (a > b) {
                        v[i] = b;
                        v[l] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// The same network by the whole block (rows longer than 256): one barrier
// per stage; len is the same in every thread.
__device__ __forceinline__ void sort_block(unsigned int* v, unsigned int len, int tid)
{
    unsigned int n2 = 1;
    while (n2 < len) n2 <<= 1;
    for (unsigned int k = 2; k <= n2; k <<= 1) {
        for (unsigned int j = k >> 1; j > 0; j >>= 1) {
            for (unsigned int i = (unsigned int)tid; i < n2; i += 256) {
                const unsigned int l = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
                if (l > i && l < len) {
                    const unsigned int a = v[i], b = v[l];
                    if (a > b) {
                        v[i] = b;
                        v[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Block b sorts the rows whose segment starts in [b RCP_RS_CAP, (b + 1)
// RCP_RS_CAP): their entries are staged in shared memory when they fit
// (RCP_RS_BUF), else sorted in place in global memory; rows of up to 32
// entries by one thread each, up to 256 by a warp each, longer ones by the
// whole block (a single warp's network over thousands of entries would be a
// long chain of dependent shared-memory steps).
__global__ void __launch_bounds__(256)
k_row_sort(const unsigned int* rowptr, long long N, const unsigned int* colu, unsigned int* col)
{
    extern __shared__ unsigned int rs_buf[];
    __shared__ unsigned int s_r[2], s_nmed, s_nlong;
    __shared__ unsigned int s_med[256], s_long[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 2) {
        // first row whose start is at or beyond the bucket's edge
        const unsigned long long edge = ((unsigned long long)blockIdx.x + (unsigned long long)tid) * RCP_RS_CAP;
        long long lo = 0, hi = N;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if ((unsigned long long)rowptr[mid] < edge) lo = mid + 1;
            else hi = mid;
        }
        s_r[tid] = (unsigned int)lo;
    }
    if (tid == 0) s_nmed = s_nlong = 0;
    __syncthreads();
    const unsigned int rlo = s_r[0], rhi = s_r[1];
    const unsigned int e0 = rowptr[rlo], e1 = rowptr[rhi];
    const bool staged = e1 - e0 <= RCP_RS_BUF;
    unsigned int* v = staged ? rs_buf : col + e0;
    for (unsigned int e = e0 + tid; e < e1; e += 256) v[e - e0] = colu[e];
    __syncthreads();
    for (unsigned int r0 = rlo; r0 < rhi; r0 += 256) {
        const unsigned int r = r0 + tid;
        if (r < rhi) {
            const unsigned int a = rowptr[r], len = rowptr[r + 1] - a;
            if (len <= 32) sort_serial(v + (a - e0), len);
            else if (len <= 256) s_med[atomicAdd(&s_nmed, 1u)] = r;
            else s_long[atomicAdd(&s_nlong, 1u)] = r;
        }
        __syncthreads();
        for (unsigned int q = warp; q < s_nmed; q += 8) {
            const unsigned int r2 = s_med[q], a = rowptr[r2];
            sort_warp(v + (a - e0), rowptr[r2 + 1] - a, lane);
        }
        for (unsigned int q = 0; q < s_nlong; ++q) {   // block-uniform loop
            const unsigned int r2 = s_long[q], a = rowptr[r2];
            __syncthreads();
            sort_block(v + (a - e0), rowptr[r2 + 1] - a, tid);
        }
        __syncthreads();
        if (tid == 0) s_nmed = s_nlong = 0;
        __syncthreads();
    }
    if (staged)
        for (unsigned int e = e0 + tid; e < e1; e += 256) col[e] = v[e - e0];
}

// Rows longer than long_row, compacted in ascending order (flags, an
// exclusive scan, then this kernel); the mixed pair kernel gives each a warp.
__global__ void k_long_flags(const unsigned int* rowptr, long long N, unsigned int long_row, unsigned int* flags)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) flags[i] = (rowptr[i + 1] - rowptr[i] > long_row) ? 1u : 0u;
}

__global__ void k_long_compact(RcpCtl* ctl, const unsigned int* flags, const unsigned int* offs, long long N,
                               unsigned int* long_rows)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (flags[i]) long_rows[offs[i]] = (unsigned int)i;
    if (i == N - 1) ctl->n_long = offs[i] + flags[i];
}

__global__ void k_build_end(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, double4_32a* xb,
                            unsigned long long P)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c.N && xb) xb[i] = (ctl->parity ? xB : xA)[i];   // no binary64 snapshot in a mixed build
    if (i == 0) {
        ctl->need_rebuild = 0;
        ctl->disp_flag = 0u;
        ctl->kbud_bits = RCP_KBUD_INF;
        ctl->rebuilds += 1;
        ctl->pairs = P;
        if (!c.canon) mix_fill(ctl, c);   // kappa_b and sigma0 changed
    }
}
