// rcp_noalloc.cu -- binary64 energy/gradient evaluation that allocates no
// memory at all.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool that
// another runtime owns and has fully reserved, embedded or real-time hosts
// whose device memory is partitioned once at start-up, or a process that
// must not touch the allocator while another library holds it.  For them this
// entry point evaluates Eq. energy, its gradient, dE/dkappa and the largest
// fractional overlap on caller-owned device buffers (positions, diameters and
// a CSR neighbour list), exactly as rcp_energy_grad does in binary64 mode,
// using only a fixed scratch area that is part of the library image.
//
// The scratch (block partial sums and one max accumulator) is a file-scope
// static __device__ array sized for at most RCP_NOALLOC_MAX_N spheres: every
// GPU that loads the library holds it (about 192 KiB) until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; later calls reuse it.
#include <mutex>

#include "rcp_internal.cuh"

#define NA_THREADS 256
#define NA_MAX_BLOCKS (RCP_NOALLOC_MAX_N / NA_THREADS)
#define NA_MAX_DEVICES 64

struct NaScratch {
    double part_e[NA_MAX_BLOCKS];  // per-block tree of e_i = sum_{j>i} eps/2 delta^2
    double part_k[NA_MAX_BLOCKS];  // per-block tree of k_i = sum_{j>i} eps delta (1-delta)/kappa
    double part_d[NA_MAX_BLOCKS];  // per-block tree of D_i^0
    unsigned long long maxdelta_bits;
};

static __device__ __align__(256) NaScratch na_scratch;

namespace {

std::mutex na_mutex;
NaScratch* na_addr[NA_MAX_DEVICES] = {nullptr};

struct NaBox {
    double L[3], h[3];
};

__device__ __forceinline__ double na_min_image(double t, double L, double h)
{
    if (t > h) t = t - L;
    else if (t < -h) t = t + L;
    return t;
}

// Pairwise tree of the values of a block's threads in thread order (adjacent
// lanes, then adjacent warps); valid in thread 0.
template <int NT>
__device__ __forceinline__ double na_block_tree(double v, double* sh)
{
    for (int o = 1; o < 32; o <<= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int s = 1; s < NT / 32; s <<= 1)
            for (int k = 0; k + s < NT / 32; k += 2 * s) sh[k] = sh[k] + sh[k + s];
        r = sh[0];
    }
    __syncthreads();
    return r;
}

__global__ void na_clear(NaScratch* s) { s->maxdelta_bits = 0ull; }

// One thread per row i of the list (ascending columns): the left fold of
// k_pair64 in gradient mode, on [N][3] positions and separate diameters.
__global__ void __launch_bounds__(NA_THREADS)
na_pair(const double* __restrict__ x, const double* __restrict__ D0, long long N, NaBox b, double kappa, double eps,
        const unsigned int* __restrict__ rowptr, const unsigned int* __restrict__ col, double* __restrict__ grad,
        NaScratch* s)
{
    __shared__ double sh[NA_THREADS / 32];
    const long long i = (long long)blockIdx.x * NA_THREADS + threadIdx.x;
    double e = 0.0, k = 0.0, md = 0.0, d0 = 0.0;
    if (i < N) {
        const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2], Di = D0[i];
        d0 = Di;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (unsigned int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            const unsigned int j = col[t];
            double dx = na_min_image(xi - x[3 * j], b.L[0], b.h[0]);
            double dy = na_min_image(yi - x[3 * j + 1], b.L[1], b.h[1]);
            double dz = na_min_image(zi - x[3 * j + 2], b.L[2], b.h[2]);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double dd = kappa * (0.5 * (Di + D0[j]));
            double delta = 1.0 - r / dd;
            if (delta > 0.0) {
                if (r > 0.0) {
                    double coef = (eps * delta) / (dd * r);
                    g0 = g0 - coef * dx;
                    g1 = g1 - coef * dy;
                    g2 = g2 - coef * dz;
                }
                if ((long long)j > i) {
                    e = e + (0.5 * eps) * (delta * delta);
                    k = k + ((eps * delta) * (1.0 - delta)) / kappa;
                }
                if (delta > md) md = delta;
            }
        }
        grad[3 * i] = g0;
        grad[3 * i + 1] = g1;
        grad[3 * i + 2] = g2;
    }
    const double se = na_block_tree<NA_THREADS>(e, sh);
    const double sk = na_block_tree<NA_THREADS>(k, sh);
    const double sd = na_block_tree<NA_THREADS>(d0, sh);
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_down_sync(0xffffffffu, md, o));
    if ((threadIdx.x & 31) == 0 && md > 0.0) atomicMax(&s->maxdelta_bits, dbits(md));
    if (threadIdx.x == 0) {
        s->part_e[blockIdx.x] = se;
        s->part_k[blockIdx.x] = sk;
        s->part_d[blockIdx.x] = sd;
    }
}

// Pairwise tree over a[lo, lo + C) (C a power of two, zero beyond n), in
// index order, with a stack of partial sums (a binary counter).
__device__ __forceinline__ double na_chunk_tree(const double* a, long long lo, long long C, long long n)
{
    double st[16];
    int lv[16];
    int top = 0;
    for (long long t = 0; t < C; ++t) {
        double v = (lo + t < n) ? a[lo + t] : 0.0;
        int l = 0;
        while (top > 0 && lv[top - 1] == l) {
            v = st[top - 1] + v;
            --top;
            ++l;
        }
        st[top] = v;
        lv[top] = l;
        ++top;
    }
    return st[0];
}

// Trees over the nb block partials, then E, dE/dkappa and max delta.
__global__ void __launch_bounds__(1024)
na_finish(NaScratch* s, long long nb, double kappa, double mu, double* E, double* dEdk, double* maxdelta)
{
    __shared__ double sh[32];
    long long M = 1;
    while (M < nb) M <<= 1;
    const long long C = M > 1024 ? M / 1024 : 1;
    const long long lo = (long long)threadIdx.x * C;
    const double te = na_block_tree<1024>(na_chunk_tree(s->part_e, lo, C, nb), sh);
    const double tk = na_block_tree<1024>(na_chunk_tree(s->part_k, lo, C, nb), sh);
    const double td = na_block_tree<1024>(na_chunk_tree(s->part_d, lo, C, nb), sh);
    if (threadIdx.x == 0) {
        if (E) *E = te - mu * (kappa * td);
        if (dEdk) *dEdk = tk - mu * td;
        if (maxdelta) *maxdelta = bitsd(s->maxdelta_bits);
    }
}

}  // namespace

extern "C" rcp_status rcp_energy_grad_noalloc(const double* x, const double* D0, long long N, const double* box,
                                              double kappa, double mu, double eps, const unsigned int* rowptr,
                                              const unsigned int* col, double* E, double* grad_x, double* dE_dkappa,
                                              double* max_delta, void* stream)
{
    if (!x || !D0 || !box || !rowptr || !col || !grad_x || N < 1) return RCP_ERR_ARG;
    if (N > RCP_NOALLOC_MAX_N) return RCP_ERR_CAPACITY;
    if (!(kappa > 0.0)) return RCP_ERR_ARG;
    NaBox b;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0)) return RCP_ERR_ARG;
        b.L[a] = box[a];
        b.h[a] = 0.5 * box[a];
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return RCP_ERR_CUDA;
    NaScratch* s = nullptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) return RCP_ERR_CUDA;
            na_addr[dev] = (NaScratch*)p;
        }
        s = na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long nb = (N + NA_THREADS - 1) / NA_THREADS;
    na_clear<<<1, 1, 0, st>>>(s);
    na_pair<<<(unsigned int)nb, NA_THREADS, 0, st>>>(x, D0, N, b, kappa, eps, rowptr, col, grad_x, s);
    na_finish<<<1, 1024, 0, st>>>(s, nb, kappa, mu, E, dE_dkappa, max_delta);
    return cudaPeekAtLastError() == cudaSuccess ? RCP_OK : RCP_ERR_CUDA;
}
