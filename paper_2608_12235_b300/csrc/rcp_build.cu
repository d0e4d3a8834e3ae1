// rcp_build.cu -- the size-stratified multilevel cell grid and the Verlet
// list (the B300 replacement of the k-d tree of App. A).
//
// Every sphere gets an interaction radius rho_i = kappa_b D_i^0 (1/2 + s) +
// sigma0 (half its diameter plus its skin); a pair is listed iff its
// minimum-image distance is below rho_i + rho_j.  Spheres are binned into
// size classes by rho (class k holds rho in (rho_max 2^-(k+1), rho_max
// 2^-k]), each class with its own uniform grid whose cell edge is at least
// the class's largest interaction diameter.  The grids are sparse: particles
// are sorted by the 62-bit key (class, cz, cy, cx) with a hand-written LSD
// radix sort, and a hash table maps each occupied cell to its range.  A
// sphere scans its own class and every coarser class over the cells within
// its search radius; a pair inside one class is found from both ends, a pair
// across classes from the finer end only, which emits both directions.  The
// pairs (row << b | col) are radix-sorted into CSR rows with ascending
// columns.  Integer and exact-predicate work only: the list is bit-identical
// to the definition.
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
        ctl->rho_lvl[k] = 0.0;
    }
    ctl->nlev = 0;
}

__global__ void k_rho(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, double* rho)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (i < c.N) {
        const double4_32a* x = ctl->parity ? xB : xA;
        r = (ctl->kappa_b * x[i].w) * (0.5 + c.skin_s) + ctl->sigma0;
        rho[i] = r;
    }
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0 && r > 0.0) atomicMax(&ctl->rho_max_bits, dbits(r));
}

// Class k_i = max{k in [0, 31] : rho_i 2^k <= rho_max} (exact power-of-two
// scaling), and the largest rho of each class.
__global__ void k_level(RcpCtl* ctl, long long N, const double* rho, int* lvl)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double rmax = bitsd(ctl->rho_max_bits);
    const double r = rho[i];
    int k = 0;
    while (k + 1 < RCP_KMAX && ldexp(r, k + 1) <= rmax) ++k;
    lvl[i] = k;
    atomicMax(&ctl->rho_lvl_bits[k], dbits(r));
}

// Cells per axis of each class: the largest power of two n <= 2^19 with
// L/n >= 2 rho_max(k).  Also the periodic-image rule: every listed pair must
// be closer than half a box edge, i.e. 4 rho_max < min L.
__global__ void k_grid(RcpCtl* ctl, RcpConst c)
{
    int nlev = 0;
    for (int k = 0; k < RCP_KMAX; ++k) {
        double r = bitsd(ctl->rho_lvl_bits[k]);
        ctl->rho_lvl[k] = r;
        for (int a = 0; a < 3; ++a) {
            unsigned int n = 1;
            if (r > 0.0)
                while (n < RCP_NMAX_AXIS && c.L[a] / (double)(2 * n) >= 2.0 * r) n *= 2;
            ctl->ng[k][a] = (int)n;
        }
        if (r > 0.0) nlev = k + 1;
    }
    ctl->nlev = nlev;
    const double rmax = bitsd(ctl->rho_max_bits);
    if (!(4.0 * rmax < c.Lmin)) {
        ctl->status = RCP_ERR_IMAGE;
        ctl->halted = 1;
    }
}

__device__ __forceinline__ unsigned int cell_of(double x, double L, unsigned int n)
{
    double f = floor((x / L) * (double)n);
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
                           unsigned long long* key, unsigned int* idx)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double4_32a* x = ctl->parity ? xB : xA;
    const double4_32a p = x[i];
    const int k = lvl[i];
    unsigned int cx = cell_of(p.x, c.L[0], (unsigned int)ctl->ng[k][0]);
    unsigned int cy = cell_of(p.y, c.L[1], (unsigned int)ctl->ng[k][1]);
    unsigned int cz = cell_of(p.z, c.L[2], (unsigned int)ctl->ng[k][2]);
    key[i] = pack_key((unsigned int)k, cz, cy, cx);
    idx[i] = (unsigned int)i;
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  Pass = histogram per block of
// RCP_SORT_THREADS * RCP_SORT_ITEMS keys (digit-major layout), exclusive scan
// over (digit, block), stable scatter.
#define RCP_TILE (RCP_SORT_THREADS * RCP_SORT_ITEMS)

__global__ void __launch_bounds__(RCP_SORT_THREADS)
k_radix_hist(const unsigned long long* keys, long long n, int shift, unsigned int* hist, unsigned int nblocks)
{
    __shared__ unsigned int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RCP_TILE;
    for (int j = 0; j < RCP_SORT_ITEMS; ++j) {
        long long t = base + (long long)j * RCP_SORT_THREADS + threadIdx.x;
        if (t < n) atomicAdd(&cnt[(unsigned int)(keys[t] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(unsigned long long)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: within a block, keys are placed in (chunk, warp, lane)
// order; ranks inside a warp come from __match_any_sync.
__global__ void __launch_bounds__(RCP_SORT_THREADS)
k_radix_scatter(const unsigned long long* keys, const unsigned int* vals, long long n, int shift,
                const unsigned int* hist, unsigned int nblocks, unsigned long long* okeys, unsigned int* ovals)
{
    constexpr int NW = RCP_SORT_THREADS / 32;
    __shared__ unsigned int base[256];
    __shared__ unsigned int wc[NW][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = hist[(unsigned long long)tid * nblocks + blockIdx.x];
    for (int w = 0; w < NW; ++w) wc[w][tid] = 0;
    __syncthreads();
    const unsigned int lt = (1u << lane) - 1u;
    const long long tile = (long long)blockIdx.x * RCP_TILE;
    for (int j = 0; j < RCP_SORT_ITEMS; ++j) {
        const long long t = tile + (long long)j * RCP_SORT_THREADS + tid;
        const bool valid = t < n;
        const unsigned long long key = valid ? keys[t] : 0ull;
        const unsigned int val = (valid && vals) ? vals[t] : 0u;
        const unsigned int digit = valid ? ((unsigned int)(key >> shift) & 255u) : 256u;
        const unsigned int peers = __match_any_sync(0xffffffffu, digit);
        const unsigned int rank = __popc(peers & lt);
        if (valid && rank == 0) wc[warp][digit] = __popc(peers);
        __syncthreads();
        {
            unsigned int run = base[tid];
            for (int w = 0; w < NW; ++w) {
                unsigned int cc = wc[w][tid];
                wc[w][tid] = run;
                run += cc;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const unsigned int pos = wc[warp][digit] + rank;
            okeys[pos] = key;
            if (vals) ovals[pos] = val;
        }
        __syncthreads();
        for (int w = 0; w < NW; ++w) wc[w][tid] = 0;
        __syncthreads();
    }
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
// Open-addressing hash of occupied cells: key -> [start, end) in the sorted
// order.  Linear probing; the table has at least twice as many slots as
// spheres, so an empty slot always ends a probe sequence.
__device__ __forceinline__ unsigned long long hmix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_hash_heads(const unsigned long long* keys, long long n, unsigned long long* hkeys, uint2* hvals,
                             unsigned long long hmask)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned long long key = keys[t];
    const bool head = (t == 0) || keys[t - 1] != key;
    const bool tail = (t == n - 1) || keys[t + 1] != key;
    if (!head && !tail) return;
    unsigned long long s = hmix(key) & hmask;
    for (unsigned long long probe = 0; probe <= hmask; ++probe) {
        unsigned long long prev = atomicCAS(&hkeys[s], RCP_HASH_EMPTY, key);
        if (prev == RCP_HASH_EMPTY || prev == key) {
            if (head) hvals[s].x = (unsigned int)t;
            if (tail) hvals[s].y = (unsigned int)(t + 1);
            return;
        }
        s = (s + 1) & hmask;
    }
}

__device__ __forceinline__ bool hfind(const unsigned long long* hkeys, const uint2* hvals, unsigned long long hmask,
                                      unsigned long long key, uint2& out)
{
    unsigned long long s = hmix(key) & hmask;
    for (unsigned long long probe = 0; probe <= hmask; ++probe) {
        const unsigned long long k = hkeys[s];
        if (k == key) {
            out = hvals[s];
            return true;
        }
        if (k == RCP_HASH_EMPTY) return false;
        s = (s + 1) & hmask;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Pair search.  fill = 0: count the entries sphere i emits; fill = 1: write
// them at offs[i].  The inclusion test is the exact binary64 predicate
//   dx^2 + dy^2 + dz^2 < (rho_i + rho_j)^2   (minimum image).
__global__ void __launch_bounds__(256)
k_search(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const double* rho, const int* lvl,
         const unsigned int* idx_sorted, const unsigned long long* hkeys, const uint2* hvals,
         unsigned long long hmask, const unsigned int* offs, unsigned int* cnt, unsigned long long* pairs,
         int fill, int nbits)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double4_32a* x = ctl->parity ? xB : xA;
    const double4_32a xi = x[i];
    const double ri = rho[i];
    const int li = lvl[i];
    const double pi3[3] = {xi.x, xi.y, xi.z};
    unsigned int count = 0;
    unsigned long long w = fill ? offs[i] : 0ull;
    for (int k = 0; k <= li; ++k) {
        const double rk = ctl->rho_lvl[k];
        if (!(rk > 0.0)) continue;
        const double R = (ri + rk) + 1e-9 * c.Lmax;
        long long lo[3];
        unsigned int nc[3], ng[3];
        for (int a = 0; a < 3; ++a) {
            ng[a] = (unsigned int)ctl->ng[k][a];
            long long l = (long long)floor(((pi3[a] - R) / c.L[a]) * (double)ng[a]);
            long long h = (long long)floor(((pi3[a] + R) / c.L[a]) * (double)ng[a]);
            if (h - l + 1 >= (long long)ng[a]) {
                lo[a] = 0;
                nc[a] = ng[a];
            } else {
                lo[a] = l;
                nc[a] = (unsigned int)(h - l + 1);
            }
        }
        for (unsigned int cz = 0; cz < nc[2]; ++cz) {
            const unsigned int z = (unsigned int)((lo[2] + cz) & (long long)(ng[2] - 1));
            for (unsigned int cy = 0; cy < nc[1]; ++cy) {
                const unsigned int y = (unsigned int)((lo[1] + cy) & (long long)(ng[1] - 1));
                for (unsigned int cx = 0; cx < nc[0]; ++cx) {
                    const unsigned int xx = (unsigned int)((lo[0] + cx) & (long long)(ng[0] - 1));
                    uint2 range;
                    if (!hfind(hkeys, hvals, hmask, pack_key((unsigned int)k, z, y, xx), range)) continue;
                    for (unsigned int t = range.x; t < range.y; ++t) {
                        const unsigned int j = idx_sorted[t];
                        if ((long long)j == i) continue;
                        const double4_32a xj = x[j];
                        double dx = min_image_b(xi.x - xj.x, c.L[0], c.halfL[0]);
                        double dy = min_image_b(xi.y - xj.y, c.L[1], c.halfL[1]);
                        double dz = min_image_b(xi.z - xj.z, c.L[2], c.halfL[2]);
                        double r2 = dx * dx + dy * dy + dz * dz;
                        double cut = ri + rho[j];
                        if (!(r2 < cut * cut)) continue;
                        if (fill) {
                            pairs[w++] = ((unsigned long long)i << nbits) | j;
                            if (k < li) pairs[w++] = ((unsigned long long)j << nbits) | (unsigned long long)i;
                        } else {
                            count += (k < li) ? 2u : 1u;
                        }
                    }
                }
            }
        }
    }
    if (!fill) cnt[i] = count;
}

// CSR from the sorted pair keys: columns are the low bits; rowptr[i] is the
// first entry of row i (binary search), rowptr[N] = P.
__global__ void k_csr(const unsigned long long* pairs, long long P, long long N, int nbits, unsigned int* rowptr,
                      unsigned int* col)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long mask = (1ull << nbits) - 1ull;
    if (t < P) col[t] = (unsigned int)(pairs[t] & mask);
    if (t <= N) {
        const unsigned long long key = (unsigned long long)t << nbits;
        long long lo = 0, hi = P;
        while (lo < hi) {
            long long mid = lo + (hi - lo) / 2;
            if (pairs[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        rowptr[t] = (unsigned int)lo;
    }
}

__global__ void k_build_end(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, double4_32a* xb,
                            unsigned long long P)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c.N) xb[i] = (ctl->parity ? xB : xA)[i];
    if (i == 0) {
        ctl->need_rebuild = 0;
        ctl->disp_flag = 0u;
        ctl->rebuilds += 1;
        ctl->pairs = P;
    }
}
