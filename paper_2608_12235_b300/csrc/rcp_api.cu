// rcp_api.cu -- the C ABI (include/rcp.h): handle life cycle, the
// neighbour-structure build, evaluation, the standalone Adam step, and the
// host-side schedule controller that launches a captured CUDA graph whose
// device-side loop runs `chunk` iterations per body pass until one halts.
//
// Scalar schedule values (mu, learning rates, rung budgets) are computed on
// the host from device-reduced sums, in the same binary64 expressions as the
// definition (compiled with -ffp-contract=off); every per-particle and
// per-pair operation runs in the kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rcp_internal.cuh"

namespace {

struct Rung {
    double dstar, lrs;
    long long budget;
    int final_rung;
};

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct rcp_ctx {
    long long N = 0;
    long long n_mobile = 0;   // spheres Adam moves (N minus the frozen ones)
    rcp_config cfg;
    RcpConst c;
    unsigned long long seed = 0;
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    char err[512] = {0};

    // state
    double* D0 = nullptr;
    double4_32a* xA = nullptr;
    double4_32a* xB = nullptr;
    double4_32a* xb = nullptr;
    double* m64 = nullptr;
    double* v64 = nullptr;
    float* m32 = nullptr;
    float* v32 = nullptr;
    MixRec* rA = nullptr;   // mixed-precision pair records (double-buffered)
    MixRec* rB = nullptr;
    MixRec* rb = nullptr;   // records at the last build
    double* g = nullptr;      // [3N] gradient output / input buffer
    double* part_e = nullptr; // block partials
    double* row_e = nullptr;  // binary64 warp-per-row kernel: e_i and k_i of every row
    double* row_k = nullptr;
    double* part_k = nullptr;
    double* part_e2 = nullptr;
    double* part_k2 = nullptr;
    double* xtmp = nullptr;   // [3N] staging for host copies
    RcpCtl* ctl = nullptr;
    RcpCtl* ctl_h = nullptr;  // pinned mirror

    // neighbour structure
    double* rho = nullptr;
    float4* xf = nullptr;    // binary32 copy (x/L, rho) for the search prefilter
    float4* xsf = nullptr;   // the same in cell order
    int* lvl = nullptr;
    unsigned long long* key = nullptr;
    unsigned long long* key1 = nullptr;
    unsigned long long* key2 = nullptr;
    unsigned int* idx1 = nullptr;
    unsigned int* idx2 = nullptr;
    const unsigned int* idx_sorted = nullptr;
    const unsigned long long* skeys = nullptr;  // sorted cell keys of the last build
    // mixed path: the state is kept in cell-key order; perm[i] is the caller's
    // index of internal sphere i (NULL in binary64 mode: caller order)
    unsigned int* perm = nullptr;
    unsigned int* perm_alt = nullptr;
    double* D0_alt = nullptr;
    double* rho_alt = nullptr;
    int* lvl_alt = nullptr;
    uint2* cells = nullptr;             // dense cell table of all size classes
    unsigned long long cells_cap = 0;
    unsigned int* cnt = nullptr;   // [N+1]
    unsigned int* offs = nullptr;  // [N+1]
    unsigned long long* pairs1 = nullptr;
    unsigned long long* pairs2 = nullptr;
    unsigned int* col = nullptr;
    unsigned int* rowptr = nullptr;  // [N+1]
    unsigned int* long_rows = nullptr;  // [N] rows longer than RCP_LONG_ROW
    uint2* sheavy = nullptr;            // [N] search windows queued for a warp each (sphere, class)
    unsigned long long pcap = 0;
    unsigned int* cptr = nullptr;       // cell row pointers of the counting sort [ncells + 1]
    unsigned int* ccnt = nullptr;       // per-cell counts, then fill cursors [ncells + 1]
    unsigned int* scan_tmp = nullptr;
    unsigned long long scan_tmp_cap = 0;
    bool built = false;
    bool placing = false;        // placement rounds: build_b ends with the conflict search
    unsigned char* place_flags = nullptr;   // placement: sphere placed
    unsigned char* place_reject = nullptr;  // placement: candidate gives way this round
    int place_class = 0;         // placement: the size class being placed
    int place_rounds_used = 0;
    unsigned long long P = 0;

    // schedule
    std::vector<Rung> rungs;
    int rung = -1;
    long long rung_start = 0;
    double kappa_rung = 0.0;
    double SD = 0, SD3 = 0, SD4 = 0, Dref = 0, Neff = 0, kappa0 = 0, sigma0 = 0;
    double mu = 0, eta_x = 0, eta_k = 0;

    // kernel launches issued (a replayed graph counts each of its kernels)
    long long launches = 0;
    long long g_kernels = 0;

    // graph (captured on cap_stream: the user stream, or the handle's own
    // stream when the user stream is the legacy default stream, which cannot
    // be captured -- replays are then ordered with events)
    cudaGraphExec_t gexec = nullptr;
    int gT = 0;
    cudaStream_t g_stream = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    unsigned long long g_pcap = 0;
};

namespace {

rcp_status fail(rcp_ctx* h, rcp_status s, const char* fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(h, e_ == cudaErrorMemoryAllocation ? RCP_ERR_OOM : RCP_ERR_CUDA,      \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKS(expr)                       \
    do {                                \
        rcp_status s_ = (expr);         \
        if (s_ != RCP_OK) return s_;    \
    } while (0)

#define CKL()  CK(cudaPeekAtLastError())

template <typename T>
rcp_status dalloc(rcp_ctx* h, T** p, size_t count)
{
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (count == 0) count = 1;
    CK(cudaMalloc((void**)p, sizeof(T) * count));
    return RCP_OK;
}

int bits_for(unsigned long long v)  // bits needed to hold values < v (at least 1)
{
    int b = 1;
    while (b < 63 && (1ull << b) < v) ++b;
    return b;
}

rcp_status sync_ctl(rcp_ctx* h)
{
    CK(cudaMemcpyAsync(h->ctl_h, h->ctl, sizeof(RcpCtl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RCP_OK;
}

// Mixed precision keeps positions in the fixed-point records; write their
// binary64 view into the current position buffer before a binary64 consumer.
rcp_status materialize(rcp_ctx* h)
{
    if (h->cfg.precision != RCP_MIXED) return RCP_OK;
    h->launches += 1;
    k_from_fixed<<<rcp_ceil_div(h->N, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->rA, h->rB, h->D0, h->xA, h->xB);
    CK(cudaPeekAtLastError());
    return RCP_OK;
}

// The caller's index of every internal sphere, to the host (identity in
// binary64 mode).
rcp_status copy_perm(rcp_ctx* h, unsigned int* out)
{
    const size_t n = (size_t)h->N;
    if (!h->perm) {
        for (size_t i = 0; i < n; ++i) out[i] = (unsigned int)i;
        return RCP_OK;
    }
    CK(cudaMemcpyAsync(out, h->perm, sizeof(unsigned int) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RCP_OK;
}

// Tree sum of f(D0) (power 1, 3 or 4) into *dst (device), canonical order.
rcp_status tree_sum_D(rcp_ctx* h, int power, double* dst)
{
    long long n = h->N;
    unsigned int nb = rcp_ceil_div(n, RCP_TREE);
    h->launches += 1;
    k_tree_terms<<<nb, RCP_TREE, 0, h->stream>>>(h->D0, n, power, h->part_e);
    CKL();
    double* a = h->part_e;
    double* b = h->part_e2;
    n = nb;
    while (n > 1) {
        nb = rcp_ceil_div(n, RCP_TREE);
        h->launches += 1;
        k_tree_pass<<<nb, RCP_TREE, 0, h->stream>>>(a, n, b);
        CKL();
        std::swap(a, b);
        n = nb;
    }
    CK(cudaMemcpyAsync(dst, a, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return RCP_OK;
}

// ---------------------------------------------------------------- scan / sort
rcp_status ensure_scan_tmp(rcp_ctx* h, unsigned long long n)
{
    // totals of every recursion level
    unsigned long long need = 0, m = n;
    while (m > 4096) {
        m = (m + 4095) / 4096;
        need += m + 1;
    }
    need += 16;
    if (need > h->scan_tmp_cap) {
        CKS(dalloc(h, &h->scan_tmp, need));
        h->scan_tmp_cap = need;
    }
    return RCP_OK;
}

// Exclusive scan of n unsigned ints (in may equal out).
rcp_status scan_u32(rcp_ctx* h, const unsigned int* in, unsigned long long n, unsigned int* out,
                    unsigned int* tmp)
{
    if (n == 0) return RCP_OK;
    unsigned int nb = rcp_ceil_div(n, 4096);
    if (nb == 1) {
        h->launches += 1;
        k_scan_block<<<1, 1024, 0, h->stream>>>(in, (long long)n, out, nullptr);
        CKL();
        return RCP_OK;
    }
    unsigned int* totals = tmp;
    h->launches += 1;
    k_scan_block<<<nb, 1024, 0, h->stream>>>(in, (long long)n, out, totals);
    CKL();
    CKS(scan_u32(h, totals, nb, totals, tmp + nb + 1));
    h->launches += 1;
    k_scan_add<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(out, (long long)n, totals);
    CKL();
    return RCP_OK;
}

// ---------------------------------------------------------------- build
rcp_status search_once(rcp_ctx* h);
rcp_status relist_long(rcp_ctx* h);

rcp_status ensure_pair_capacity(rcp_ctx* h, unsigned long long P)
{
    if (P <= h->pcap && h->pairs1) return RCP_OK;
    unsigned long long cap = P + P / 4 + 1024;
    CKS(dalloc(h, &h->pairs1, cap));
    CKS(dalloc(h, &h->pairs2, cap));
    CKS(dalloc(h, &h->col, cap));
    h->pcap = cap;
    return RCP_OK;
}

// The build runs in three phases separated by host reads, so that several
// packings can be built concurrently on their own streams (the batch):
//   A: class sizes and grids (ctl copied to the host);
//   B: keys, sort, cell table, search (entry count copied to the host);
//   C: pair sort, CSR, long-row list, snapshot.
// A mixed build (outside placement) works from the fixed-point records
// alone: radii, keys and the prefilter's copy from the records, the search's
// band positions converted where needed; no binary64 view is formed.
static bool records_build(const rcp_ctx* h) { return h->cfg.precision == RCP_MIXED && !h->placing; }

rcp_status build_a(rcp_ctx* h)
{
    const long long N = h->N;
    const unsigned int nbN = rcp_ceil_div(N, 256);
    h->launches += 1;
    k_build_begin<<<1, 1, 0, h->stream>>>(h->ctl, h->sigma0);
    h->launches += 1;
    if (records_build(h))
        k_rho_mixed<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->rA, h->rB, h->D0, h->rho, h->xf);
    else   // binary64 positions (placement writes them itself)
        k_rho<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->rho, h->xf);
    h->launches += 1;
    k_level<<<nbN, 256, 0, h->stream>>>(h->ctl, N, h->rho, h->lvl);
    h->launches += 1;
    k_grid<<<1, 128, 0, h->stream>>>(h->ctl, h->c);
    CKL();
    CK(cudaMemcpyAsync(h->ctl_h, h->ctl, sizeof(RcpCtl), cudaMemcpyDeviceToHost, h->stream));
    return RCP_OK;
}

rcp_status build_b(rcp_ctx* h)
{
    const long long N = h->N;
    const unsigned int nbN = rcp_ceil_div(N, 256);
    if (h->ctl_h->status == RCP_ERR_IMAGE)
        return fail(h, RCP_ERR_IMAGE,
                    "largest interaction diameter 4 rho_max = %.6g reaches the smallest box edge %.6g: a sphere "
                    "would meet its own periodic image",
                    4.0 * h->ctl_h->rho_lvl[0], h->c.Lmin);
    h->launches += 1;
    if (records_build(h))
        k_cell_key_mixed<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->rA, h->rB, h->lvl, h->key);
    else
        k_cell_key<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->lvl, h->key);
    CKL();
    // spheres by cell: a counting sort over the dense cell table through the
    // CSR kernels (rows = cells, each row sorted by sphere index), the order
    // of a stable sort of the cell keys
    const unsigned long long ncells = h->ctl_h->cell_off[RCP_KMAX];
    if (ncells > h->cells_cap) {
        CKS(dalloc(h, &h->cells, ncells));
        CKS(dalloc(h, &h->cptr, ncells + 1));
        CKS(dalloc(h, &h->ccnt, ncells + 1));
        CKS(ensure_scan_tmp(h, ncells + 1));
        h->cells_cap = ncells;
    }
    const int cbits = bits_for((unsigned long long)N);
    unsigned long long* ck = h->key1;
    unsigned int* colu = h->idx1;
    const unsigned int* sidx = h->idx2;
    const unsigned long long* skeys = h->key2;
    CK(cudaMemsetAsync(h->ccnt, 0, sizeof(unsigned int) * (ncells + 1), h->stream));
    h->launches += 2;
    k_cell_pairs<<<nbN, 256, 0, h->stream>>>(h->ctl, N, h->key, cbits, ck);
    k_row_count<<<nbN, 256, 0, h->stream>>>(ck, N, cbits, h->ccnt);
    CKL();
    CKS(scan_u32(h, h->ccnt, ncells + 1, h->cptr, h->scan_tmp));
    CK(cudaMemsetAsync(h->ccnt, 0, sizeof(unsigned int) * ncells, h->stream));   // fill cursors
    h->launches += 5;
    k_row_scatter<<<nbN, 256, 0, h->stream>>>(ck, N, cbits, h->cptr, h->ccnt, colu);
    k_row_sort<<<rcp_ceil_div(N, RCP_RS_CAP), 256, RCP_RS_BUF * sizeof(unsigned int), h->stream>>>(
        h->cptr, (long long)ncells, colu, h->idx2);
    k_gather_keys<<<nbN, 256, 0, h->stream>>>(N, sidx, h->key, h->key2);
    k_cell_table<<<rcp_ceil_div(ncells, 256), 256, 0, h->stream>>>(h->cptr, ncells, h->cells);
    CKL();
    h->idx_sorted = sidx;
    h->skeys = skeys;
    h->launches += 1;
    k_gather_sorted<<<nbN, 256, 0, h->stream>>>(N, h->idx_sorted, h->xf, h->xsf);
    if (h->perm && !h->placing) {
        // mixed path: move the state into cell-key order (moments through the
        // gradient buffer, which holds nothing between evaluations)
        float* m2 = reinterpret_cast<float*>(h->g);
        float* v2 = m2 + 3 * (size_t)N;
        h->launches += 2;
        k_permute_state<<<nbN, 256, 0, h->stream>>>(h->ctl, N, sidx, h->rA, h->rB, nullptr, nullptr, h->m32, h->v32, m2,
                                                    v2, h->D0, h->D0_alt, h->rho, h->rho_alt, h->lvl, h->lvl_alt,
                                                    h->perm, h->perm_alt);
        k_flip_parity<<<1, 1, 0, h->stream>>>(h->ctl);
        CKL();
        CK(cudaMemcpyAsync(h->m32, m2, sizeof(float) * 3 * (size_t)N, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(h->v32, v2, sizeof(float) * 3 * (size_t)N, cudaMemcpyDeviceToDevice, h->stream));
        std::swap(h->D0, h->D0_alt);
        std::swap(h->rho, h->rho_alt);
        std::swap(h->lvl, h->lvl_alt);
        std::swap(h->perm, h->perm_alt);
        h->idx_sorted = nullptr;   // sphere t is now the t-th in key order
    }
    return search_once(h);
}

rcp_status search_once(rcp_ctx* h)
{
    const long long N = h->N;
    const unsigned int nbN = rcp_ceil_div(N, 256);
    const int nbits = bits_for((unsigned long long)N);
    if (h->placing) {
        h->launches += 1;
        k_place_conflicts<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->rho, h->lvl, h->idx_sorted,
                                                      h->xsf, h->cells, h->D0, h->place_flags, h->place_reject,
                                                      h->place_class);
        CKL();
        return RCP_OK;
    }
    // the entry cursor and the queue of heavy windows (adjacent in RcpCtl)
    static_assert(offsetof(RcpCtl, search_heavy) == offsetof(RcpCtl, pair_cursor) + sizeof(unsigned long long),
                  "pair_cursor and search_heavy are cleared together");
    CK(cudaMemsetAsync(&h->ctl->pair_cursor, 0, sizeof(unsigned long long) + sizeof(unsigned int), h->stream));
    const unsigned int hcap = (unsigned int)N;
    h->launches += 2;
    const MixRec* rA = records_build(h) ? h->rA : nullptr;
    const MixRec* rB = records_build(h) ? h->rB : nullptr;
    k_search<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, rA, rB, h->rho, h->lvl, h->idx_sorted, h->xsf,
                                         h->cells, h->pairs1, h->pcap, nbits, h->sheavy, hcap);
    k_search_heavy<<<std::min(nbN, 8u * 148u), 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, rA, rB, h->rho,
                                                                     h->lvl, h->idx_sorted, h->xsf, h->cells,
                                                                     h->pairs1, h->pcap, nbits, h->sheavy, hcap);
    CKL();
    CK(cudaMemcpyAsync(&h->ctl_h->pair_cursor, &h->ctl->pair_cursor, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, h->stream));
    return RCP_OK;
}

rcp_status build_c(rcp_ctx* h)
{
    const long long N = h->N;
    const unsigned int nbN = rcp_ceil_div(N, 256);
    const int nbits = bits_for((unsigned long long)N);
    unsigned long long P = h->ctl_h->pair_cursor;
    if (P > h->pcap) {
        // entries beyond the old capacity were dropped: grow and search again
        CKS(ensure_pair_capacity(h, P));
        CKS(search_once(h));
        CK(cudaStreamSynchronize(h->stream));
        P = h->ctl_h->pair_cursor;
    }
    // the pair kernels step 32-bit entry indices up to 64 past the last entry
    if (P >= (1ull << 32) - 1024) return fail(h, RCP_ERR_CAPACITY, "more than 2^32 - 1024 listed pairs");
    // CSR rows: per-row counts and their scan (rowptr), every column into its
    // row's segment, each segment sorted (k_row_sort): the list a full sort
    // of the keys gives, in a fraction of the memory passes
    CK(cudaMemsetAsync(h->cnt, 0, sizeof(unsigned int) * ((size_t)N + 1), h->stream));
    if (P > 0) {
        h->launches += 1;
        k_row_count<<<rcp_ceil_div(P, 256), 256, 0, h->stream>>>(h->pairs1, (long long)P, nbits, h->cnt);
        CKL();
    }
    CKS(scan_u32(h, h->cnt, (unsigned long long)N + 1, h->rowptr, h->scan_tmp));
    if (P > 0) {
        CK(cudaMemsetAsync(h->cnt, 0, sizeof(unsigned int) * (size_t)N, h->stream));   // fill cursors
        unsigned int* colu = reinterpret_cast<unsigned int*>(h->pairs2);
        h->launches += 2;
        k_row_scatter<<<rcp_ceil_div(P, 256), 256, 0, h->stream>>>(h->pairs1, (long long)P, nbits, h->rowptr,
                                                                   h->cnt, colu);
        k_row_sort<<<rcp_ceil_div(P, RCP_RS_CAP), 256, RCP_RS_BUF * sizeof(unsigned int), h->stream>>>(
            h->rowptr, N, colu, h->col);
        CKL();
    }
    CKS(relist_long(h));
    h->launches += 1;
    k_build_end<<<nbN, 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, records_build(h) ? nullptr : h->xb, P);
    CKL();
    if (h->cfg.precision == RCP_MIXED) {
        h->launches += 1;
        k_snap_records<<<nbN, 256, 0, h->stream>>>(h->ctl, N, h->rA, h->rB, h->rb);
        CKL();
    }
    h->P = P;
    h->built = true;
    return RCP_OK;
}

// Rows longer than c.long_row, compacted (used by the mixed pair kernel).
rcp_status relist_long(rcp_ctx* h)
{
    if (h->c.long_row > 32u) h->c.long_row = 32u;   // short rows are marked in one 32-bit word
    const long long N = h->N;
    const unsigned int nbN = rcp_ceil_div(N, 256);
    h->launches += 1;
    k_long_flags<<<nbN, 256, 0, h->stream>>>(h->rowptr, N, h->c.long_row, h->cnt);
    CKL();
    CKS(scan_u32(h, h->cnt, (unsigned long long)N, h->offs, h->scan_tmp));
    h->launches += 1;
    k_long_compact<<<nbN, 256, 0, h->stream>>>(h->ctl, h->cnt, h->offs, N, h->long_rows);
    CKL();
    return RCP_OK;
}

rcp_status build(rcp_ctx* h)
{
    CKS(build_a(h));
    CK(cudaStreamSynchronize(h->stream));
    CKS(build_b(h));
    CK(cudaStreamSynchronize(h->stream));
    return build_c(h);
}

// ---------------------------------------------------------------- evaluation
unsigned int pair_blocks(const rcp_ctx* h) { return rcp_ceil_div(h->N, RCP_PAIR_THREADS); }

// Blocks of one pair-kernel launch, each writing one partial: the row
// blocks in binary64 mode (canonical trees), the long-row blocks and the
// row blocks in mixed mode.
unsigned int launch_blocks(const rcp_ctx* h)
{
    if (h->cfg.precision == RCP_MIXED) return pair_blocks(h) + h->c.long_blocks;
    return pair_blocks(h);
}

// Binary64 packings up to RCP_WARP_ROW_MAX_N spheres take a warp per row
// (k_pair64_warp), which leaves one e_i and k_i per row instead of block
// partials.
bool warp_rows(const rcp_ctx* h) { return h->c.canon && h->N <= RCP_WARP_ROW_MAX_N; }

// Reduce the pair kernel's partials a, b (n of each) to <= 8192 entries by
// tree passes over aligned groups (the canonical order); returns the buffers
// and count to hand to k_kappa_step.
void prereduce(rcp_ctx* h, const double* a, const double* b, long long n, const double** pe, const double** pk,
               long long* nb)
{
    bool flip = false;
    while (n > 8192) {
        unsigned int g = rcp_ceil_div(n, RCP_TREE);
        double* oa = flip ? h->part_e : h->part_e2;
        double* ob = flip ? h->part_k : h->part_k2;
        k_tree_pass2<<<g, RCP_TREE, 0, h->stream>>>(a, b, n, oa, ob);
        a = oa;
        b = ob;
        n = g;
        flip = !flip;
    }
    *pe = a;
    *pk = b;
    *nb = n;
}

size_t kappa_smem(long long nb)
{
    long long M = 1;
    while (M < nb) M <<= 1;
    return 2 * sizeof(double) * (size_t)M;
}

// One iteration (or one evaluation) on the stream; optional events bracket
// the pair kernel (ev[0], ev[1]) and close the iteration (ev[2]).  Returns the
// number of kernels it launched.
int launch_iteration(rcp_ctx* h, int mode, cudaEvent_t* ev = nullptr)
{
    const unsigned int nb = pair_blocks(h);
    if (ev) cudaEventRecord(ev[0], h->stream);
    if (h->cfg.precision == RCP_MIXED) {
        // a bounded packing takes the kernel with the wall terms, frozen
        // spheres (a seated stage) the one that tells their contact
        // diameters apart, the rest the plain one
        (h->c.bounded ? k_pair_mixed_wl : (h->c.nfrozen > 0 ? k_pair_mixed_fz : k_pair_mixed))<<<nb + h->c.long_blocks, RCP_PAIR_THREADS, 0, h->stream>>>(
            h->ctl, h->c, h->m32, h->v32, h->rA, h->rB, h->rowptr, h->col, h->long_rows, h->rb, h->part_e, h->part_k,
            mode, h->g);
    } else if (warp_rows(h)) {
        k_pair64_warp<<<rcp_ceil_div(h->N * 32, RCP_WARP_ROW_THREADS), RCP_WARP_ROW_THREADS, 0, h->stream>>>(
            h->ctl, h->c, h->xA, h->xB, h->m64, h->v64, h->rowptr, h->col, h->xb, h->row_e, h->row_k, mode, h->g);
    } else {
        k_pair64_long<<<RCP_LONG_BLOCKS_MAX, RCP_PAIR_THREADS, 0, h->stream>>>(
            h->ctl, h->c, h->xA, h->xB, h->m64, h->v64, h->rowptr, h->col, h->long_rows, h->xb, h->row_e, h->row_k,
            mode, h->g);
        k_pair64<<<nb, RCP_PAIR_THREADS, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->m64, h->v64, h->rowptr,
                                                          h->col, h->xb, h->part_e, h->part_k, mode, h->g, h->row_e,
                                                          h->row_k);
    }
    if (ev) cudaEventRecord(ev[1], h->stream);
    if (h->cfg.precision == RCP_MIXED) {
        // block partials as compensated binary32 pairs, reduced and closed by one kernel
        k_kappa_mixed<<<1, 1024, 0, h->stream>>>(h->ctl, h->c, h->part_e, h->part_k, (long long)launch_blocks(h), mode);
        if (ev) cudaEventRecord(ev[2], h->stream);
        return 2;
    }
    const bool wr = warp_rows(h);
    const long long n0 = wr ? h->N : (long long)launch_blocks(h);
    const double* pe;
    const double* pk;
    long long n;
    prereduce(h, wr ? h->row_e : h->part_e, wr ? h->row_k : h->part_k, n0, &pe, &pk, &n);
    k_kappa_step<<<1, 1024, kappa_smem(n), h->stream>>>(h->ctl, h->c, pe, pk, n, mode);
    if (ev) cudaEventRecord(ev[2], h->stream);
    int passes = h->c.long64 ? 1 : 0;   // k_pair64_long
    for (long long m = n0; m > 8192; m = (m + RCP_TREE - 1) / RCP_TREE) ++passes;
    return 2 + passes;
}

struct ProfileAcc {
    double ms_pair = 0.0, ms_iter = 0.0;
    long long launches = 0;
    cudaEvent_t ev[3];
};

rcp_status ensure_list(rcp_ctx* h)
{
    if (!h->built) return build(h);
    CKS(sync_ctl(h));
    if (h->ctl_h->need_rebuild) return build(h);
    return RCP_OK;
}

bool capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy; }

cudaStream_t capture_stream(const rcp_ctx* h) { return capturable(h->stream) ? h->stream : h->own_stream; }

// The replayed graph: a conditional while node whose body is `chunk`
// iterations followed by k_loop_cond, so one launch advances the packing
// until an iteration halts (a rebuild due, the rung's iteration limit, the
// stop, an error) and no launch after the halt runs empty beyond the rest of
// its body pass.
rcp_status capture_graph(rcp_ctx* h)
{
    if (h->gexec && h->gT == h->cfg.chunk && h->g_stream == h->stream && h->g_pcap == h->pcap) return RCP_OK;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle hc;
    cudaError_t e0 = cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault);
    // zeroed storage: the params type has no default constructor (a union)
    alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)];
    memset(np_buf, 0, sizeof(np_buf));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_buf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wn;
    if (e0 == cudaSuccess) e0 = cudaGraphAddNode(&wn, graph, nullptr, nullptr, 0, &np);
    if (e0 != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(h, RCP_ERR_CUDA, "graph loop node failed: %s", cudaGetErrorString(e0));
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t user = h->stream;
    h->stream = capture_stream(h);  // launch_iteration issues on h->stream
    e0 = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e0 != cudaSuccess) {
        h->stream = user;
        cudaGraphDestroy(graph);
        return fail(h, RCP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e0));
    }
    h->g_kernels = 1;
    for (int t = 0; t < h->cfg.chunk; ++t) h->g_kernels += launch_iteration(h, RCP_MODE_ADAM);
    k_loop_cond<<<1, 1, 0, h->stream>>>(h->ctl, hc);
    cudaGraph_t captured;
    cudaError_t e = cudaStreamEndCapture(h->stream, &captured);
    h->stream = user;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(h, RCP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    h->gT = h->cfg.chunk;
    h->g_stream = h->stream;
    h->g_pcap = h->pcap;
    return RCP_OK;
}

// ---------------------------------------------------------------- schedule
// Rung table (reading of App. A): rung 0 lasts n_trig of Eq. trigger, every
// later rung n_trig/4, both at least n_min; the target overlap falls tenfold
// and the learning rate halves per rung of the descent; then n_cycles
// cycles raise mu one decade and lower it back; the final rung has mu = 0,
// half the learning rate, and runs until the stopping criterion.
void build_rungs(rcp_ctx* h)
{
    const rcp_config& p = h->cfg;
    double nt = (4000.0 * (double)p.Y + (double)p.X * std::sqrt((double)(h->n_mobile * (long long)h->c.dim))) - 2000.0;
    long long b0 = (long long)std::ceil(nt);
    if (b0 < p.n_min) b0 = p.n_min;
    long long bq = (long long)std::ceil(nt / 4.0);
    if (bq < p.n_min) bq = p.n_min;
    h->rungs.clear();
    double ds = p.delta_star0, lrs = 1.0;
    h->rungs.push_back({ds, lrs, b0, 0});
    for (int r = 1; r <= p.n_down; ++r) {
        ds = ds / 10.0;
        lrs = lrs * 0.5;
        h->rungs.push_back({ds, lrs, bq, 0});
    }
    for (int cy = 0; cy < p.n_cycles; ++cy) {
        h->rungs.push_back({ds * 10.0, lrs, bq, 0});
        h->rungs.push_back({ds, lrs, bq, 0});
    }
    h->rungs.push_back({0.0, lrs * 0.5, p.max_iters, 1});
}

// Values of rung r given kappa at its start:
//   mu = 3 delta* eps N_eff / (kappa_r sum D^0),  N_eff = sum D^3 / D_ref^3,
//   eta_x = lr_x lrs kappa_r D_ref,  eta_kappa = lr_kappa lrs kappa_r.
void rung_values(rcp_ctx* h, int r, double kr)
{
    const Rung& R = h->rungs[r];
    h->mu = R.dstar > 0.0 ? (((3.0 * R.dstar) * h->cfg.eps) * h->Neff) / (kr * h->SD) : 0.0;
    h->eta_x = ((h->cfg.lr_x * R.lrs) * kr) * h->Dref;
    h->eta_k = (h->cfg.lr_kappa * R.lrs) * kr;
}

}  // namespace

// ============================================================================
extern "C" {

rcp_status rcp_config_default(rcp_config* cfg)
{
    if (!cfg) return RCP_ERR_ARG;
    memset(cfg, 0, sizeof(*cfg));
    cfg->precision = RCP_FP64;
    cfg->phi0 = 0.05;
    cfg->eps = 1.0;
    cfg->beta1 = 0.9;
    cfg->beta2 = 0.999;
    cfg->adam_eps = 1e-8;
    cfg->skin_s = 0.1;
    cfg->skin_theta = 1.0;
    cfg->skin_abs = 20.0;
    cfg->lr_x = 1e-3;
    cfg->lr_kappa = 1e-3;
    cfg->delta_star0 = 1e-2;
    cfg->tol = 5e-4;
    cfg->Y = 2;
    cfg->X = 9;
    cfg->n_min = 2000;
    cfg->n_down = 3;
    cfg->n_cycles = 2;
    cfg->max_iters = 2000000;
    cfg->chunk = 32;
    cfg->cell_occupancy = 1.0;
    cfg->placement = 0;
    cfg->place_rounds = 10000;
    return RCP_OK;
}

const char* rcp_status_str(rcp_status s)
{
    switch (s) {
    case RCP_OK: return "ok";
    case RCP_ERR_ARG: return "invalid argument";
    case RCP_ERR_IMAGE: return "periodic-image rule violated";
    case RCP_ERR_OOM: return "out of device memory";
    case RCP_ERR_NAN: return "non-finite energy or gradient";
    case RCP_ERR_CAPACITY: return "internal capacity exceeded";
    case RCP_ERR_TIMEOUT: return "device wait timed out";
    case RCP_ERR_MAXITER: return "iteration cap reached";
    case RCP_ERR_CUDA: return "CUDA runtime error";
    case RCP_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* rcp_last_error(rcp_handle h) { return h ? h->err : ""; }

long long rcp_size(rcp_handle h) { return h ? h->N : 0; }

int rcp_dim(rcp_handle h) { return h ? h->c.dim : 0; }

rcp_status rcp_destroy(rcp_handle h)
{
    if (!h) return RCP_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    void* ptrs[] = {h->D0, h->xA, h->xB, h->xb, h->m64, h->v64, h->m32, h->v32, h->rA, h->rB, h->rb, h->g, h->part_e, h->part_k, h->part_e2, h->part_k2, h->xtmp, h->ctl, h->rho,
                    h->lvl, h->xf, h->xsf, h->key, h->key1, h->key2, h->idx1, h->idx2, h->cells, h->cnt,
                    h->offs, h->pairs1, h->pairs2, h->col, h->rowptr, h->long_rows, h->sheavy, h->cptr, h->ccnt, h->scan_tmp, h->perm, h->perm_alt, h->D0_alt, h->rho_alt,
                    h->lvl_alt, h->row_e, h->row_k};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->ctl_h) cudaFreeHost(h->ctl_h);
    if (h->ev_a) cudaEventDestroy(h->ev_a);
    if (h->ev_b) cudaEventDestroy(h->ev_b);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return RCP_OK;
}
// Non-overlapping placement at kappa_0 (rcp_config.placement = 1): random
// sequential addition by size class, largest class first, each class in
// rounds.  A round draws candidates for the class's spheres not yet placed
// (k_place_draw), finds every overlap of a candidate with a placed sphere or
// a class-mate's candidate with the neighbour search at rho = kappa_0 D^0 / 2
// (no skin; only candidates search), marks the candidate that gives way
// (k_place_conflicts) and keeps the rest (k_place_accept).  Runs before any
// build, in the caller's order.
rcp_status place_nonoverlapping(rcp_ctx* h, unsigned long long seed)
{
    const long long N = h->N;
    const unsigned int nbN = rcp_ceil_div(N, 256);
    unsigned char *placed = nullptr, *reject = nullptr;
    CK(cudaMalloc((void**)&placed, (size_t)N));
    if (cudaMalloc((void**)&reject, (size_t)N) != cudaSuccess) {
        cudaFree(placed);
        return fail(h, RCP_ERR_OOM, "placement flags");
    }
    h->place_flags = placed;
    h->place_reject = reject;
    const double skin_s = h->c.skin_s, sigma0 = h->sigma0;
    h->c.skin_s = 0.0;   // interaction radius rho = kappa_0 D^0 / 2
    h->sigma0 = 0.0;
    h->placing = true;
    rcp_status st = [&]() -> rcp_status {
        CK(cudaMemsetAsync(placed, 0, (size_t)N, h->stream));
        // frozen spheres are in place before any class is drawn
        if (h->c.nfrozen > 0) CK(cudaMemsetAsync(placed, 1, (size_t)h->c.nfrozen, h->stream));
        CKS(build_a(h));   // the classes (they depend on D^0 and kappa_0 only)
        CK(cudaStreamSynchronize(h->stream));
        const int nlev = h->ctl_h->nlev;
        unsigned long long counts[RCP_KMAX];
        for (int k = 0; k < RCP_KMAX; ++k) counts[k] = h->ctl_h->lvl_count[k];
        int worst = 0;
        for (int k = 0; k < nlev; ++k) {
            unsigned long long left = counts[k];
            int r = 0;
            for (; r < h->cfg.place_rounds && left > 0; ++r) {
                h->launches += 1;
                k_place_draw<<<nbN, 256, 0, h->stream>>>(seed, N, r, k, h->c, h->D0, h->lvl, placed, reject, h->xA);
                CKL();
                h->place_class = k;
                CKS(build_a(h));
                CK(cudaStreamSynchronize(h->stream));
                CKS(build_b(h));   // ends with the conflict search of class k
                CK(cudaMemsetAsync(&h->ctl->pair_cursor, 0, sizeof(unsigned long long), h->stream));
                h->launches += 1;
                k_place_accept<<<nbN, 256, 0, h->stream>>>(h->ctl, N, k, h->lvl, placed, reject);
                CKL();
                CK(cudaMemcpyAsync(&left, &h->ctl->pair_cursor, sizeof(left), cudaMemcpyDeviceToHost, h->stream));
                CK(cudaStreamSynchronize(h->stream));
            }
            if (left > 0)
                return fail(h, RCP_ERR_CAPACITY,
                            "%llu spheres of size class %d still overlap after %d placement rounds (phi0 too high?)",
                            left, k, r);
            if (r > worst) worst = r;
        }
        h->place_rounds_used = worst;
        return RCP_OK;
    }();
    h->c.skin_s = skin_s;
    h->sigma0 = sigma0;
    h->placing = false;
    h->built = false;
    h->place_flags = h->place_reject = nullptr;
    cudaFree(placed);
    cudaFree(reject);
    return st;
}


}  // extern "C"

namespace {

// Creation of a packing of Nf frozen spheres (contact diameters fixed_d,
// positions fixed_x [Nf][d]; internal indices 0..Nf-1) and Nm mobile ones
// (relative diameters `diameters`; indices Nf..).  Nf = 0 is rcp_create.
rcp_status create_impl(const double* fixed_d, const double* fixed_x, long long Nf, const double* diameters,
                       long long Nm, int d, const double* box, unsigned long long seed, const rcp_config* cfg,
                       rcp_handle* out)
{
    if (!out) return RCP_ERR_ARG;
    *out = nullptr;
    if (!diameters || !box || Nm < 1 || Nf < 0 || (Nf > 0 && (!fixed_d || !fixed_x))) return RCP_ERR_ARG;
    if (d != 2 && d != 3) return RCP_ERR_UNSUPPORTED;
    if (Nf >= (1LL << 31) || Nm >= (1LL << 31) - Nf) return RCP_ERR_ARG;
    if (cfg && (cfg->walls & ~((1 << d) - 1))) return RCP_ERR_ARG;   // one bit per axis of the caller
    if (cfg && (cfg->container < 0 || cfg->container > 2 || (cfg->container == 2 && d != 3))) return RCP_ERR_ARG;
    const long long N = Nf + Nm;
    for (long long i = 0; i < Nf; ++i) {
        if (!(fixed_d[i] > 0.0) || !std::isfinite(fixed_d[i])) return RCP_ERR_ARG;
        for (int a = 0; a < d; ++a)
            if (!std::isfinite(fixed_x[(size_t)d * i + a])) return RCP_ERR_ARG;
    }
    for (int a = 0; a < d; ++a)
        if (!(box[a] > 0.0) || !std::isfinite(box[a])) return RCP_ERR_ARG;
    // d = 2: disks held in the plane z = L_z / 2 of a box whose third edge is
    // the larger of the two (every z difference is exactly zero)
    const double box3[3] = {box[0], box[1], d == 3 ? box[2] : (box[0] > box[1] ? box[0] : box[1])};
    box = box3;
    for (long long i = 0; i < Nm; ++i)
        if (!(diameters[i] > 0.0) || !std::isfinite(diameters[i])) return RCP_ERR_ARG;
    // device encoding: -F for a frozen sphere, D^0 for a mobile one
    std::vector<double> Dh((size_t)N);
    for (long long i = 0; i < Nf; ++i) Dh[(size_t)i] = -fixed_d[i];
    for (long long i = 0; i < Nm; ++i) Dh[(size_t)(Nf + i)] = diameters[i];
    rcp_ctx* h = new rcp_ctx();
    if (cfg) h->cfg = *cfg;
    else rcp_config_default(&h->cfg);
    if (h->cfg.chunk < 1) h->cfg.chunk = 1;
    if ((h->cfg.precision != RCP_FP64 && h->cfg.precision != RCP_MIXED) || !(h->cfg.phi0 > 0.0) ||
        !(h->cfg.skin_theta > 0.0 && h->cfg.skin_theta <= 1.0) || !(h->cfg.skin_s >= 0.0) || !(h->cfg.tol > 0.0)) {
        delete h;
        return RCP_ERR_ARG;
    }
    h->N = N;
    h->n_mobile = Nm;
    h->seed = seed;
    RcpConst& c = h->c;
    memset(&c, 0, sizeof(c));
    c.N = N;
    c.nfrozen = Nf;
    c.Lmin = box[0];
    c.Lmax = box[0];
    c.walls = h->cfg.walls;
    c.container = h->cfg.container;
    // the container: a ball over the caller's axes (a disk when d = 2) or a
    // cylinder about z, radius min L_a / 2 over its axes, about the centre
    c.caxes = c.container == 1 ? (1 << d) - 1 : (c.container == 2 ? 3 : 0);
    c.bounded = c.walls | c.caxes;
    for (int a = 0; a < 3; ++a) {
        c.L[a] = box[a];
        c.halfL[a] = 0.5 * box[a];
        // a mixed record covers a periodic axis once (the integer wrap is the
        // minimum image) and a bounded one twice over, from -L/2 (a sphere
        // pushed past a wall stays representable)
        const bool bnd = (c.bounded >> a) & 1;
        c.qspan[a] = bnd ? 2.0 * box[a] : box[a];
        c.qoff[a] = bnd ? -0.5 * box[a] : 0.0;
        c.qo_hi[a] = (float)c.qoff[a];
        c.qo_lo[a] = (float)(c.qoff[a] - (double)c.qo_hi[a]);
        c.qscale[a] = (float)(c.qspan[a] * 0x1.0p-32);
        c.qinv[a] = (float)(0x1.0p32 / c.qspan[a]);
        c.invL[a] = 1.0 / box[a];
        c.invLf[a] = (float)c.invL[a];
        {
            int ex = 0;
            if (std::frexp(box[a], &ex) == 0.5) c.pow2L |= 1 << a;
        }
        {
            const double sc = c.qspan[a] * 0x1.0p-32;
            c.qs_hi[a] = (float)sc;
            c.qs_lo[a] = (float)(sc - (double)c.qs_hi[a]);
        }
        c.Lf[a] = (float)box[a];
        c.Llo[a] = (float)(box[a] - (double)c.Lf[a]);
        if (box[a] < c.Lmin) c.Lmin = box[a];
        if (box[a] > c.Lmax) c.Lmax = box[a];
    }
    // two fixed-point units of the coarsest axis: covers the remainders the
    // mixed pre-test leaves out (below one unit per axis, sqrt(3) in all)
    c.qmargin = 2.0f * std::max(c.qscale[0], std::max(c.qscale[1], c.qscale[2]));
    c.V = d == 2 ? box[0] * box[1] : (box[0] * box[1]) * box[2];   // area when d = 2
    c.Rc = INFINITY;
    for (int a = 0; a < d; ++a)
        if (((c.caxes >> a) & 1) && 0.5 * box[a] < c.Rc) c.Rc = 0.5 * box[a];
    c.wmargin = (float)(c.Lmax * 0x1.0p-20);
    c.Rc_hi = std::isfinite(c.Rc) ? (float)c.Rc : 0.0f;
    c.Rc_lo = std::isfinite(c.Rc) ? (float)(c.Rc - (double)c.Rc_hi) : 0.0f;
    if (c.container == 1) c.Vs = d == 2 ? (RCP_PI * c.Rc) * c.Rc : (((4.0 / 3.0) * RCP_PI) * ((c.Rc * c.Rc) * c.Rc));
    else if (c.container == 2) c.Vs = ((RCP_PI * c.Rc) * c.Rc) * box[2];
    else c.Vs = c.V;
    // the periodic-image rule concerns the periodic axes of the caller only
    c.Lmin = INFINITY;
    for (int a = 0; a < d; ++a)
        if (!((c.bounded >> a) & 1) && box[a] < c.Lmin) c.Lmin = box[a];
    c.dim = d;
    c.eps = h->cfg.eps;
    c.beta1 = h->cfg.beta1;
    c.beta2 = h->cfg.beta2;
    c.adam_eps = h->cfg.adam_eps;
    c.skin_s = h->cfg.skin_s;
    c.skin_theta = h->cfg.skin_theta;
    c.stop_margin = h->cfg.precision == RCP_MIXED ? 1e-2 : 0.0;
    c.cell_occ = h->cfg.cell_occupancy > 0.0 ? h->cfg.cell_occupancy : 1.0;
    c.canon = h->cfg.precision == RCP_FP64 ? 1u : 0u;
    c.long_row = RCP_LONG_ROW;
    c.long64 = (c.canon && N > RCP_WARP_ROW_MAX_N) ? 1 : 0;
    {
        // blocks serving long rows: about one per 1536 spheres, at least 2
        long long lb = N / RCP_LONG_DIV;
        if (lb < 2) lb = 2;
        if (lb > RCP_LONG_BLOCKS_MAX) lb = RCP_LONG_BLOCKS_MAX;
        c.long_blocks = (unsigned int)lb;
    }

    rcp_status st = [&]() -> rcp_status {
        CK(cudaGetDevice(&h->device));
        CK(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
        h->stream = h->own_stream;
        CK(cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming));
        const size_t n = (size_t)N;
        CKS(dalloc(h, &h->D0, n));
        CKS(dalloc(h, &h->xA, n));
        CKS(dalloc(h, &h->xB, n));
        CKS(dalloc(h, &h->xb, n));
        if (h->cfg.precision == RCP_MIXED) {
            CKS(dalloc(h, &h->m32, 3 * n));
            CKS(dalloc(h, &h->v32, 3 * n));
            CKS(dalloc(h, &h->rA, n));
            CKS(dalloc(h, &h->rB, n));
            CKS(dalloc(h, &h->rb, n));
            CKS(dalloc(h, &h->perm, n));
            CKS(dalloc(h, &h->perm_alt, n));
            CKS(dalloc(h, &h->D0_alt, n));
            CKS(dalloc(h, &h->rho_alt, n));
            CKS(dalloc(h, &h->lvl_alt, n));
            k_iota<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>((long long)n, h->perm);
            CK(cudaMemsetAsync(h->m32, 0, sizeof(float) * 3 * n, h->stream));
            CK(cudaMemsetAsync(h->v32, 0, sizeof(float) * 3 * n, h->stream));
        } else {
            CKS(dalloc(h, &h->m64, 3 * n));
            CKS(dalloc(h, &h->v64, 3 * n));
            // e_i, k_i of the rows a warp evaluates: every row of a small
            // packing, the long rows of a large one
            CKS(dalloc(h, &h->row_e, n));
            CKS(dalloc(h, &h->row_k, n));
            CK(cudaMemsetAsync(h->m64, 0, sizeof(double) * 3 * n, h->stream));
            CK(cudaMemsetAsync(h->v64, 0, sizeof(double) * 3 * n, h->stream));
        }
        CKS(dalloc(h, &h->g, 3 * n));
        CKS(dalloc(h, &h->xtmp, 3 * n));
        size_t nparts = (n + RCP_TREE - 1) / RCP_TREE +
                        ((n + RCP_PAIR_THREADS - 1) / RCP_PAIR_THREADS + RCP_LONG_BLOCKS_MAX) * (RCP_PAIR_THREADS / 32) +
                        8;
        CKS(dalloc(h, &h->part_e, nparts));
        CKS(dalloc(h, &h->part_k, nparts));
        CKS(dalloc(h, &h->part_e2, nparts));
        CKS(dalloc(h, &h->part_k2, nparts));
        CKS(dalloc(h, &h->ctl, 1));
        CK(cudaMallocHost((void**)&h->ctl_h, sizeof(RcpCtl)));
        CKS(dalloc(h, &h->rho, n));
        CKS(dalloc(h, &h->xf, n));
        CKS(dalloc(h, &h->xsf, n));
        CKS(dalloc(h, &h->lvl, n));
        CKS(dalloc(h, &h->key, n));
        CKS(dalloc(h, &h->key1, n));
        CKS(dalloc(h, &h->key2, n));
        CKS(dalloc(h, &h->idx1, n));
        CKS(dalloc(h, &h->idx2, n));
        CKS(dalloc(h, &h->cnt, n + 1));
        CKS(dalloc(h, &h->offs, n + 1));
        CKS(dalloc(h, &h->rowptr, n + 1));
        CKS(dalloc(h, &h->long_rows, n));
        CKS(dalloc(h, &h->sheavy, n));
        CKS(ensure_pair_capacity(h, 16 * (unsigned long long)n));
        CK(cudaFuncSetAttribute(k_kappa_step, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 8192 * 8));
        CKS(ensure_scan_tmp(h, n + 1));

        // control block
        RcpCtl init;
        memset(&init, 0, sizeof(init));
        init.b1 = 1.0;
        init.b2 = 1.0;
        init.need_rebuild = 1;
        init.halted = 1;
        init.shrink_bits = 0x7FF0000000000000ull;
        init.iter_limit = 0;
        CK(cudaMemcpyAsync(h->ctl, &init, sizeof(RcpCtl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->D0, Dh.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        const unsigned int nb = rcp_ceil_div(N, 256);
        h->launches += 1;
        k_init_positions<<<nb, 256, 0, h->stream>>>(seed, N, c, h->D0, h->xA);
        CKL();
        if (Nf > 0) {   // the frozen spheres where the caller holds them
            CK(cudaMemcpyAsync(h->xtmp, fixed_x, sizeof(double) * d * (size_t)Nf, cudaMemcpyHostToDevice, h->stream));
            h->launches += 1;
            k_set_positions<<<rcp_ceil_div(Nf, 256), 256, 0, h->stream>>>(Nf, c, h->xtmp, h->D0, h->xA, nullptr);
            CKL();
        }
        CKS(tree_sum_D(h, 1, &h->ctl->SD));
        CKS(tree_sum_D(h, 3, &h->ctl->SD3));
        if (d == 2) CKS(tree_sum_D(h, 2, &h->ctl->SD2));
        CKS(tree_sum_D(h, 4, &h->ctl->SD4));
        if (Nf > 0) {
            CKS(tree_sum_D(h, -3, &h->ctl->SF3));
            if (d == 2) CKS(tree_sum_D(h, -2, &h->ctl->SF2));
        }
        h->launches += 1;
        k_kappa0<<<1, 1, 0, h->stream>>>(h->ctl, h->cfg.phi0, c.Vs, d);
        CKL();
        CKS(sync_ctl(h));
        h->SD = h->ctl_h->SD;
        h->SD3 = h->ctl_h->SD3;
        h->SD4 = h->ctl_h->SD4;
        h->kappa0 = h->ctl_h->kappa;
        h->Dref = h->SD4 / h->SD3;
        h->Neff = h->SD3 / ((h->Dref * h->Dref) * h->Dref);
        h->sigma0 = h->cfg.skin_abs * ((h->cfg.lr_x * h->kappa0) * h->Dref);
        build_rungs(h);
        if (h->cfg.placement == 1) CKS(place_nonoverlapping(h, seed));
        if (h->cfg.precision == RCP_MIXED) {
            h->launches += 1;
            k_to_fixed<<<nb, 256, 0, h->stream>>>(h->ctl, c, h->xA, h->xB, h->rA, h->rB, nullptr);
            CKL();
        }
        return RCP_OK;
    }();
    if (st != RCP_OK) {
        rcp_destroy(h);
        return st;
    }
    *out = h;
    return RCP_OK;
}

}  // namespace

extern "C" {

rcp_status rcp_create(const double* diameters, long long N, int d, const double* box, unsigned long long seed,
                      const rcp_config* cfg, rcp_handle* out)
{
    return create_impl(nullptr, nullptr, 0, diameters, N, d, box, seed, cfg, out);
}

rcp_status rcp_create_seated(const double* fixed_d, const double* fixed_x, long long Nf, const double* diameters,
                             long long N, int d, const double* box, unsigned long long seed, const rcp_config* cfg,
                             rcp_handle* out)
{
    if (Nf < 1) return RCP_ERR_ARG;
    if (out) *out = nullptr;
    return create_impl(fixed_d, fixed_x, Nf, diameters, N, d, box, seed, cfg, out);
}

long long rcp_frozen(rcp_handle h) { return h ? h->c.nfrozen : 0; }

// The sequential cascade (Sec. IV) through the calls above: stage 0 packs
// class 0; stage s seats class s among the packed spheres (frozen at their
// contact diameters, seed + s), runs it to the stop, shrinks it, then
// releases all of them (a packing of the contact diameters, phi0 = the seated
// phi, kappa set to 1, placement off) and runs and shrinks that.
rcp_status rcp_cascade(const double* diameters, const int* cls, long long N, int d, const double* box,
                       unsigned long long seed, const rcp_config* cfg, double* x_out, double* diam_out,
                       double* phi_out, long long* iters_out)
{
    if (!diameters || !cls || !box || N < 1 || !x_out || !diam_out) return RCP_ERR_ARG;
    int C = 0;
    for (long long i = 0; i < N; ++i) {
        if (cls[i] < 0) return RCP_ERR_ARG;
        if (cls[i] + 1 > C) C = cls[i] + 1;
    }
    std::vector<std::vector<long long>> members((size_t)C);
    for (long long i = 0; i < N; ++i) members[(size_t)cls[i]].push_back(i);
    for (int s = 0; s < C; ++s)
        if (members[(size_t)s].empty()) return RCP_ERR_ARG;
    std::vector<long long> order;   // caller index of each packed sphere, stage order
    std::vector<double> diam, xs;    // their contact diameters and positions
    rcp_stop stop = {0, 0.0, 1};
    int slot = 0;
    auto finish = [&](rcp_handle h, const rcp_result& r, long long n) -> rcp_status {
        if (!r.stopped) return RCP_ERR_MAXITER;
        xs.assign((size_t)(n * d), 0.0);
        rcp_status st = rcp_state(h, xs.data(), nullptr, nullptr, nullptr);
        if (st != RCP_OK) return st;
        if (phi_out) phi_out[slot] = r.phi;
        if (iters_out) iters_out[slot] = r.iters;
        ++slot;
        return RCP_OK;
    };
    for (int s = 0; s < C; ++s) {
        const std::vector<long long>& nw = members[(size_t)s];
        std::vector<double> Dn(nw.size());
        for (size_t t = 0; t < nw.size(); ++t) Dn[t] = diameters[nw[t]];
        const long long nn = (long long)nw.size();
        rcp_handle h = nullptr;
        rcp_result r;
        rcp_status st;
        if (s == 0) {
            st = rcp_create(Dn.data(), nn, d, box, seed, cfg, &h);
            if (st == RCP_OK) st = rcp_run(h, &stop, &r);
            if (st == RCP_OK) st = finish(h, r, nn);
            rcp_destroy(h);
            if (st != RCP_OK) return st;
            order = nw;
            diam.resize(Dn.size());
            for (size_t t = 0; t < Dn.size(); ++t) diam[t] = r.kappa_c * Dn[t];
            continue;
        }
        const long long nf = (long long)diam.size();
        st = rcp_create_seated(diam.data(), xs.data(), nf, Dn.data(), nn, d, box, seed + (unsigned long long)s, cfg,
                               &h);
        if (st == RCP_OK) st = rcp_run(h, &stop, &r);
        if (st == RCP_OK) st = finish(h, r, nf + nn);
        rcp_destroy(h);
        if (st != RCP_OK) return st;
        for (size_t t = 0; t < Dn.size(); ++t) diam.push_back(r.kappa_c * Dn[t]);
        order.insert(order.end(), nw.begin(), nw.end());
        rcp_config rc = *cfg;
        rc.phi0 = r.phi;
        rc.placement = 0;
        h = nullptr;
        st = rcp_create(diam.data(), nf + nn, d, box, seed + (unsigned long long)s, &rc, &h);
        if (st == RCP_OK) st = rcp_set_positions(h, xs.data(), 1.0, 0);
        if (st == RCP_OK) st = rcp_run(h, &stop, &r);
        if (st == RCP_OK) st = finish(h, r, nf + nn);
        rcp_destroy(h);
        if (st != RCP_OK) return st;
        for (double& v : diam) v = r.kappa_c * v;
    }
    for (size_t t = 0; t < order.size(); ++t) {
        diam_out[order[t]] = diam[t];
        for (int a = 0; a < d; ++a) x_out[(size_t)d * order[t] + a] = xs[(size_t)d * t + a];
    }
    return RCP_OK;
}

rcp_status rcp_set_stream(rcp_handle h, void* stream)
{
    if (!h) return RCP_ERR_ARG;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own_stream;
    if (s != h->stream) {
        CK(cudaStreamSynchronize(h->stream));
        h->stream = s;
    }
    return RCP_OK;
}

rcp_status rcp_set_positions(rcp_handle h, const double* x, double kappa, int on_device)
{
    if (!h || !x) return RCP_ERR_ARG;
    const size_t n = (size_t)h->N;
    const size_t nd = (size_t)h->c.dim * n;
    if (on_device) CK(cudaMemcpyAsync(h->xtmp, x, sizeof(double) * nd, cudaMemcpyDeviceToDevice, h->stream));
    else CK(cudaMemcpyAsync(h->xtmp, x, sizeof(double) * nd, cudaMemcpyHostToDevice, h->stream));
    CKS(sync_ctl(h));
    double4_32a* cur = h->ctl_h->parity ? h->xB : h->xA;
    h->launches += 1;
    k_set_positions<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->N, h->c, h->xtmp, h->D0, cur, h->perm);
    CKL();
    if (kappa > 0.0) CK(cudaMemcpyAsync(&h->ctl->kappa, &kappa, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (h->cfg.precision == RCP_MIXED) {
        h->launches += 1;
        k_to_fixed<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->rA, h->rB, nullptr);
        CKL();
    }
    if (h->built) {
        if (h->cfg.precision == RCP_MIXED) {
            // the binary64 build snapshot from the records' snapshot
            h->launches += 1;
            k_from_fixed<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->rb, h->rb, h->D0, h->xb, h->xb);
        }
        h->launches += 1;
        k_disp_check<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->xb);
        CKL();
    }
    CK(cudaStreamSynchronize(h->stream));
    return RCP_OK;
}

rcp_status rcp_build_neighbors(rcp_handle h)
{
    if (!h) return RCP_ERR_ARG;
    CKS(build(h));
    CK(cudaStreamSynchronize(h->stream));
    return RCP_OK;
}

rcp_status rcp_energy_grad(rcp_handle h, double mu, double* E, double* grad_x, double* dE_dkappa,
                           double* max_delta, int on_device)
{
    if (!h) return RCP_ERR_ARG;
    CKS(ensure_list(h));
    // evaluation mode: mu from the argument, no iteration limit involved
    h->launches += 1;
    k_set_rung<<<1, 1, 0, h->stream>>>(h->ctl, h->c, mu, 0.0, 0.0, h->cfg.tol, 1LL << 62, 0);
    CKL();
    h->launches += launch_iteration(h, RCP_MODE_GRAD);
    CKL();
    const size_t n = (size_t)h->N;
    const double* gsrc = h->g;
    const size_t nd = (size_t)h->c.dim * n;
    if ((h->perm || h->c.dim != 3) && grad_x) {
        // internal order and layout -> the caller's
        h->launches += 1;
        k_perm3<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->N, h->c, h->perm, h->g, h->xtmp, 1);
        CKL();
        gsrc = h->xtmp;
    }
    if (on_device) {
        if (grad_x) CK(cudaMemcpyAsync(grad_x, gsrc, sizeof(double) * nd, cudaMemcpyDeviceToDevice, h->stream));
        if (E) CK(cudaMemcpyAsync(E, &h->ctl->E, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        if (dE_dkappa) CK(cudaMemcpyAsync(dE_dkappa, &h->ctl->dEdk, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        if (max_delta) CK(cudaMemcpyAsync(max_delta, &h->ctl->maxdelta, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        return RCP_OK;
    }
    if (grad_x) CK(cudaMemcpyAsync(grad_x, gsrc, sizeof(double) * nd, cudaMemcpyDeviceToHost, h->stream));
    CKS(sync_ctl(h));
    if (h->ctl_h->status == RCP_ERR_NAN) return fail(h, RCP_ERR_NAN, "non-finite energy or gradient");
    if (E) *E = h->ctl_h->E;
    if (dE_dkappa) *dE_dkappa = h->ctl_h->dEdk;
    if (max_delta) *max_delta = h->ctl_h->maxdelta;
    return RCP_OK;
}

rcp_status rcp_energy_grad_at(rcp_handle h, const double* x_dev, const double* kappa_dev, double mu, double* E,
                              double* grad_x, double* dE_dkappa, double* max_delta)
{
    if (!h || !x_dev || !kappa_dev) return RCP_ERR_ARG;
    const size_t n = (size_t)h->N;
    CK(cudaMemcpyAsync(h->xtmp, x_dev, sizeof(double) * h->c.dim * n, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(&h->ctl->kappa, kappa_dev, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->launches += 1;   // into the current buffer, chosen on the device (no host read of the parity)
    k_set_positions<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->N, h->c, h->xtmp, h->D0, h->xA, h->perm,
                                                                  h->ctl, h->xB);
    CKL();
    if (h->cfg.precision == RCP_MIXED) {
        h->launches += 1;
        k_to_fixed<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->rA, h->rB, nullptr);
        CKL();
    }
    if (h->built) {
        if (h->cfg.precision == RCP_MIXED) {
            // the binary64 build snapshot from the records' snapshot
            h->launches += 1;
            k_from_fixed<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->rb, h->rb, h->D0, h->xb, h->xb);
        }
        h->launches += 1;
        k_disp_check<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->xb);
        CKL();
    }
    return rcp_energy_grad(h, mu, E, grad_x, dE_dkappa, max_delta, 1);
}

rcp_status rcp_adam_step(rcp_handle h, const double* grad_x, double dE_dkappa, double lr_x, double lr_kappa,
                         int on_device)
{
    if (!h || !grad_x) return RCP_ERR_ARG;
    const size_t n = (size_t)h->N;
    if (!h->built) CKS(build(h));   // before the copy: a build uses h->g as scratch
    CK(cudaMemcpyAsync(h->g, grad_x, sizeof(double) * h->c.dim * n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    const double* gin = h->g;
    if (h->perm || h->c.dim != 3) {
        // the caller's order and layout -> internal
        h->launches += 1;
        k_perm3<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->N, h->c, h->perm, h->g, h->xtmp, 0);
        CKL();
        gin = h->xtmp;
    }
    h->launches += 1;
    if (h->cfg.precision == RCP_MIXED)
        k_adam_mixed<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->rA, h->rB, h->m32, h->v32, gin,
                                                                  h->rb, lr_x);
    else
        k_adam64<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->m64, h->v64, gin,
                                                               h->xb, lr_x);
    CKL();
    h->launches += 1;
    k_adam_kappa<<<1, 1, 0, h->stream>>>(h->ctl, h->c, dE_dkappa, lr_kappa);
    CKL();
    CK(cudaStreamSynchronize(h->stream));
    return RCP_OK;
}

static rcp_status do_shrink(rcp_ctx* h)
{
    CKS(ensure_list(h));
    CKS(materialize(h));
    unsigned long long inf = 0x7FF0000000000000ull;
    CK(cudaMemcpyAsync(&h->ctl->shrink_bits, &inf, sizeof(inf), cudaMemcpyHostToDevice, h->stream));
    h->launches += 1;
    k_shrink<<<pair_blocks(h), RCP_PAIR_THREADS, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->rowptr, h->col);
    h->launches += 1;
    k_shrink_final<<<1, 1, 0, h->stream>>>(h->ctl, h->c);
    CKL();
    return sync_ctl(h);
}

rcp_status rcp_shrink(rcp_handle h, double* kappa_c, double* phi)
{
    if (!h) return RCP_ERR_ARG;
    CKS(do_shrink(h));
    if (kappa_c) *kappa_c = h->ctl_h->kappa_c;
    if (phi) *phi = h->ctl_h->phi;
    return RCP_OK;
}

static void fill_result(rcp_ctx* h, rcp_result* out, double secs, long long launches)
{
    if (!out) return;
    out->launches = launches;
    const RcpCtl* c = h->ctl_h;
    out->iters = c->iter;
    out->rebuilds = c->rebuilds;
    out->pairs = (long long)c->pairs;
    out->stopped = c->stopped;
    out->kappa = c->kappa;
    out->max_delta = c->maxdelta;
    out->energy = c->E;
    out->kappa_c = c->kappa_c;
    out->phi = c->phi;
    out->seconds = secs;
}

static rcp_status verify_stop_mixed(rcp_ctx* h, bool* stop);

static rcp_status run_impl(rcp_ctx* h, const rcp_stop* stop, rcp_result* out, ProfileAcc* prof)
{
    auto t0 = std::chrono::steady_clock::now();
    rcp_stop st = {0, 0.0, 1};
    if (stop) st = *stop;
    CKS(sync_ctl(h));
    const long long call_start = h->ctl_h->iter;
    const long long launches0 = h->launches;
    rcp_status result = RCP_OK;
    for (;;) {
        RcpCtl* hc = h->ctl_h;
        if (hc->stopped) {
            if (st.shrink) CKS(do_shrink(h));
            break;
        }
        if (h->rung < 0) {
            h->rung = 0;
            h->rung_start = hc->iter;
            h->kappa_rung = hc->kappa;
        }
        const Rung& R = h->rungs[h->rung];
        long long rung_end = R.final_rung ? h->cfg.max_iters : h->rung_start + R.budget;
        if (rung_end > h->cfg.max_iters) rung_end = h->cfg.max_iters;
        if (hc->iter >= rung_end) {
            if (R.final_rung || hc->iter >= h->cfg.max_iters) {
                result = fail(h, RCP_ERR_MAXITER, "iteration cap %lld reached before the stopping criterion",
                              h->cfg.max_iters);
                break;
            }
            h->rung += 1;
            h->rung_start = hc->iter;
            h->kappa_rung = hc->kappa;
            continue;
        }
        long long limit = rung_end;
        if (st.max_iters > 0 && call_start + st.max_iters < limit) limit = call_start + st.max_iters;
        if (prof && hc->iter + 1 < limit) limit = hc->iter + 1;
        if (hc->iter >= limit) break;
        if (st.max_seconds > 0.0) {
            double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (secs >= st.max_seconds) break;
        }
        rung_values(h, h->rung, h->kappa_rung);
        if (!h->built || hc->need_rebuild) CKS(build(h));
        if (!prof) CKS(capture_graph(h));
        h->launches += 1;
        k_set_rung<<<1, 1, 0, h->stream>>>(h->ctl, h->c, h->mu, h->eta_x, h->eta_k, h->cfg.tol, limit, R.final_rung);
        CKL();
        if (prof) {
            h->launches += launch_iteration(h, RCP_MODE_ADAM, prof->ev);
            CKL();
            CK(cudaEventSynchronize(prof->ev[2]));
            float a = 0.f, b = 0.f;
            CK(cudaEventElapsedTime(&a, prof->ev[0], prof->ev[1]));
            CK(cudaEventElapsedTime(&b, prof->ev[0], prof->ev[2]));
            prof->ms_pair += a;
            prof->ms_iter += b;
            prof->launches += 1;
        } else {
            const cudaStream_t cs = capture_stream(h);
            if (cs != h->stream) {
                CK(cudaEventRecord(h->ev_a, h->stream));
                CK(cudaStreamWaitEvent(cs, h->ev_a, 0));
            }
            const unsigned long long passes0 = hc->body_passes;
            CK(cudaGraphLaunch(h->gexec, cs));
            if (cs != h->stream) {
                CK(cudaEventRecord(h->ev_b, cs));
                CK(cudaStreamWaitEvent(h->stream, h->ev_b, 0));
            }
            CKS(sync_ctl(h));
            h->launches += (long long)(h->ctl_h->body_passes - passes0) * h->g_kernels;
        }
        if (prof) CKS(sync_ctl(h));
        hc = h->ctl_h;
        if (hc->status != RCP_OK) {
            result = fail(h, (rcp_status)hc->status, "device status %d (%s) at iteration %lld", hc->status,
                          rcp_status_str((rcp_status)hc->status), hc->iter);
            break;
        }
        if (hc->verify) {
            bool s = false;
            CKS(verify_stop_mixed(h, &s));
        }
    }
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    fill_result(h, out, secs, h->launches - launches0);
    return result;
}

rcp_status rcp_run(rcp_handle h, const rcp_stop* stop, rcp_result* out)
{
    if (!h) return RCP_ERR_ARG;
    return run_impl(h, stop, out, nullptr);
}

rcp_status rcp_profile(rcp_handle h, long long iters, double* ms_pair, double* ms_iter, long long* launches)
{
    if (!h || iters < 1) return RCP_ERR_ARG;
    ProfileAcc acc;
    for (int e = 0; e < 3; ++e) CK(cudaEventCreate(&acc.ev[e]));
    rcp_stop st = {iters, 0.0, 0};
    rcp_status s = run_impl(h, &st, nullptr, &acc);
    for (int e = 0; e < 3; ++e) cudaEventDestroy(acc.ev[e]);
    if (ms_pair) *ms_pair = acc.ms_pair;
    if (ms_iter) *ms_iter = acc.ms_iter;
    if (launches) *launches = acc.launches;
    return s;
}

static rcp_status verify_stop_mixed(rcp_ctx* h, bool* stop)
{
    // binary64 maximum overlap of the state that the binary32 pass flagged
    CKS(materialize(h));
    h->launches += 1;
    k_maxdelta64<<<pair_blocks(h), RCP_PAIR_THREADS, 0, h->stream>>>(h->ctl, h->c, h->xA, h->xB, h->rowptr,
                                                                      h->col);
    h->launches += 1;
    k_verify_final<<<1, 1, 0, h->stream>>>(h->ctl, h->c);
    CKL();
    CKS(sync_ctl(h));
    *stop = h->ctl_h->stopped != 0;
    return RCP_OK;
}

rcp_status rcp_state(rcp_handle h, double* x, double* m, double* v, rcp_scalars* s)
{
    if (!h) return RCP_ERR_ARG;
    CKS(sync_ctl(h));
    const size_t n = (size_t)h->N;
    const int dc = h->c.dim;
    if (x) {
        CKS(materialize(h));
        const double4_32a* cur = h->ctl_h->parity ? h->xB : h->xA;
        h->launches += 1;
        k_get_positions<<<rcp_ceil_div(n, 256), 256, 0, h->stream>>>(h->N, h->c, cur, h->xtmp, h->perm);
        CKL();
        CK(cudaMemcpyAsync(x, h->xtmp, sizeof(double) * h->c.dim * n, cudaMemcpyDeviceToHost, h->stream));
    }
    if (h->cfg.precision == RCP_MIXED) {
        std::vector<float> tmp(m || v ? 3 * n : 0);
        std::vector<unsigned int> pm(m || v ? n : 0);
        if (m || v) CKS(copy_perm(h, pm.data()));
        if (m) {
            CK(cudaMemcpyAsync(tmp.data(), h->m32, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < n; ++i)
                for (int a = 0; a < dc; ++a) m[dc * (size_t)pm[i] + a] = tmp[3 * i + a];
        }
        if (v) {
            CK(cudaMemcpyAsync(tmp.data(), h->v32, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < n; ++i)
                for (int a = 0; a < dc; ++a) v[dc * (size_t)pm[i] + a] = tmp[3 * i + a];
        }
    } else {
        if (dc == 3) {
            if (m) CK(cudaMemcpyAsync(m, h->m64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
            if (v) CK(cudaMemcpyAsync(v, h->v64, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
        } else {
            std::vector<double> tmp(m || v ? 3 * n : 0);
            for (int w = 0; w < 2; ++w) {
                double* out = w == 0 ? m : v;
                if (!out) continue;
                CK(cudaMemcpyAsync(tmp.data(), w == 0 ? h->m64 : h->v64, sizeof(double) * 3 * n,
                                   cudaMemcpyDeviceToHost, h->stream));
                CK(cudaStreamSynchronize(h->stream));
                for (size_t i = 0; i < n; ++i)
                    for (int a = 0; a < dc; ++a) out[dc * i + a] = tmp[3 * i + a];
            }
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    if (s) {
        const RcpCtl* c = h->ctl_h;
        s->t = c->iter;
        s->kappa = c->kappa;
        s->m_kappa = c->mk;
        s->v_kappa = c->vk;
        s->b1 = c->b1;
        s->b2 = c->b2;
        s->rung = h->rung;
        s->rung_start = h->rung_start;
        s->kappa_rung = h->kappa_rung;
        s->stopped = c->stopped;
    }
    return RCP_OK;
}

rcp_status rcp_load_state(rcp_handle h, const double* x, const double* m, const double* v, const rcp_scalars* s)
{
    if (!h) return RCP_ERR_ARG;
    const size_t n = (size_t)h->N;
    const int dc = h->c.dim;
    if (x) CKS(rcp_set_positions(h, x, s ? s->kappa : 0.0, 0));
    if (h->cfg.precision == RCP_MIXED) {
        std::vector<float> tmp(3 * n);
        std::vector<unsigned int> pm(m || v ? n : 0);
        if (m || v) CKS(copy_perm(h, pm.data()));
        if (m) {
            for (size_t i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) tmp[3 * i + a] = a < dc ? (float)m[dc * (size_t)pm[i] + a] : 0.0f;
            CK(cudaMemcpyAsync(h->m32, tmp.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
        if (v) {
            for (size_t i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) tmp[3 * i + a] = a < dc ? (float)v[dc * (size_t)pm[i] + a] : 0.0f;
            CK(cudaMemcpyAsync(h->v32, tmp.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    } else {
        if (dc == 3) {
            if (m) CK(cudaMemcpyAsync(h->m64, m, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
            if (v) CK(cudaMemcpyAsync(h->v64, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
        } else {
            std::vector<double> tmp(3 * n);
            for (int w = 0; w < 2; ++w) {
                const double* in = w == 0 ? m : v;
                if (!in) continue;
                for (size_t i = 0; i < n; ++i)
                    for (int a = 0; a < 3; ++a) tmp[3 * i + a] = a < dc ? in[dc * i + a] : 0.0;
                CK(cudaMemcpyAsync(w == 0 ? h->m64 : h->v64, tmp.data(), sizeof(double) * 3 * n,
                                   cudaMemcpyHostToDevice, h->stream));
                CK(cudaStreamSynchronize(h->stream));
            }
        }
    }
    if (s) {
        CKS(sync_ctl(h));
        RcpCtl c = *h->ctl_h;
        c.iter = s->t;
        c.kappa = s->kappa;
        c.mk = s->m_kappa;
        c.vk = s->v_kappa;
        c.b1 = s->b1;
        c.b2 = s->b2;
        c.stopped = s->stopped;
        c.halted = 1;
        c.need_rebuild = 1;
        CK(cudaMemcpyAsync(h->ctl, &c, sizeof(RcpCtl), cudaMemcpyHostToDevice, h->stream));
        h->rung = s->rung;
        h->rung_start = s->rung_start;
        h->kappa_rung = s->kappa_rung;
    }
    CK(cudaStreamSynchronize(h->stream));
    return RCP_OK;
}

rcp_status rcp_neighbors(rcp_handle h, long long* rowptr, int* col, long long cap, long long* P)
{
    if (!h || !rowptr || !P) return RCP_ERR_ARG;
    if (!h->built) CKS(build(h));
    const size_t n = (size_t)h->N;
    std::vector<unsigned int> rp(n + 1);
    CK(cudaMemcpyAsync(rp.data(), h->rowptr, sizeof(unsigned int) * (n + 1), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *P = (long long)h->P;
    const bool want_col = col && (long long)h->P <= cap;
    if (!h->perm) {
        for (size_t i = 0; i <= n; ++i) rowptr[i] = rp[i];
        if (want_col) {
            CK(cudaMemcpyAsync(col, h->col, sizeof(unsigned int) * h->P, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
        return RCP_OK;
    }
    // mixed path: rows and columns are internal indices; return the list in
    // the caller's order, columns ascending per row
    std::vector<unsigned int> pm(n), inv(n), cs(want_col ? h->P : 0);
    CKS(copy_perm(h, pm.data()));
    if (want_col) {
        CK(cudaMemcpyAsync(cs.data(), h->col, sizeof(unsigned int) * h->P, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    for (size_t i = 0; i < n; ++i) inv[pm[i]] = (unsigned int)i;
    rowptr[0] = 0;
    for (size_t u = 0; u < n; ++u) {
        const size_t r = inv[u];
        const unsigned int len = rp[r + 1] - rp[r];
        if (want_col) {
            int* out = col + rowptr[u];
            for (unsigned int t = 0; t < len; ++t) out[t] = (int)pm[cs[rp[r] + t]];
            std::sort(out, out + len);
        }
        rowptr[u + 1] = rowptr[u] + len;
    }
    return RCP_OK;
}

rcp_status rcp_cell_keys(rcp_handle h, unsigned long long* keys)
{
    if (!h || !keys) return RCP_ERR_ARG;
    if (!h->built) CKS(build(h));
    const size_t n = (size_t)h->N;
    if (!h->perm) {
        CK(cudaMemcpyAsync(keys, h->key, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return RCP_OK;
    }
    // mixed path: internal sphere t holds the t-th sorted key
    std::vector<unsigned long long> sk(n);
    std::vector<unsigned int> pm(n);
    CK(cudaMemcpyAsync(sk.data(), h->skeys, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, h->stream));
    CKS(copy_perm(h, pm.data()));
    for (size_t t = 0; t < n; ++t) keys[pm[t]] = sk[t];
    return RCP_OK;
}

}  // extern "C"

// ============================================================================
// Batches: many independent packings advanced by one graph of batched
// kernels.  Each packing keeps its own handle (state, list, schedule); the
// batched pair kernel and kappa step walk a device array of per-packing
// descriptors, block b serving packing p with local block b - bstart[p], so
// a packing computes exactly what its own launch would (bit-identical
// trajectories).  Packings stop, pause and rebuild independently; rebuilds
// of several packings run concurrently on their own streams.

namespace {

enum PlanResult { PLAN_RUN, PLAN_PAUSE, PLAN_STOPPED, PLAN_MAXITER, PLAN_ERROR };

// Next replay of one packing from h->ctl_h (iter, kappa, stopped, status):
// the rung logic of rcp_run.
PlanResult plan_replay(rcp_ctx* h, long long call_start, long long call_max, long long* limit, int* final_rung)
{
    RcpCtl* hc = h->ctl_h;
    if (hc->status != RCP_OK) return PLAN_ERROR;
    if (hc->stopped) return PLAN_STOPPED;
    if (h->rung < 0) {
        h->rung = 0;
        h->rung_start = hc->iter;
        h->kappa_rung = hc->kappa;
    }
    long long rung_end = 0;
    for (;;) {
        const Rung& R = h->rungs[h->rung];
        rung_end = R.final_rung ? h->cfg.max_iters : h->rung_start + R.budget;
        if (rung_end > h->cfg.max_iters) rung_end = h->cfg.max_iters;
        if (hc->iter < rung_end) break;
        if (R.final_rung || hc->iter >= h->cfg.max_iters) return PLAN_MAXITER;
        h->rung += 1;
        h->rung_start = hc->iter;
        h->kappa_rung = hc->kappa;
    }
    long long lim = rung_end;
    if (call_max > 0 && call_start + call_max < lim) lim = call_start + call_max;
    if (hc->iter >= lim) return PLAN_PAUSE;
    rung_values(h, h->rung, h->kappa_rung);
    *limit = lim;
    *final_rung = h->rungs[h->rung].final_rung;
    return PLAN_RUN;
}

PackDev pack_of(rcp_ctx* h)
{
    PackDev q;
    memset(&q, 0, sizeof(q));
    q.ctl = h->ctl;
    q.c = h->c;
    q.c.long64 = 0;   // the batched binary64 kernel walks every row itself
    q.xA = h->xA;
    q.xB = h->xB;
    q.xb = h->xb;
    q.m64 = h->m64;
    q.v64 = h->v64;
    q.m32 = h->m32;
    q.v32 = h->v32;
    q.rA = h->rA;
    q.rB = h->rB;
    q.rb = h->rb;
    q.rowptr = h->rowptr;
    q.col = h->col;
    q.long_rows = h->long_rows;
    q.part_e = h->part_e;
    q.part_k = h->part_k;
    q.g = h->g;
    q.nparts = launch_blocks(h);
    q.nblocks = pair_blocks(h) + (h->cfg.precision == RCP_MIXED ? h->c.long_blocks : 0);
    return q;
}

}  // namespace

struct rcp_batch_ctx {
    int B = 0;
    std::vector<rcp_ctx*> hs;
    int precision = 0;
    cudaStream_t stream = nullptr;
    PackDev* d_packs = nullptr;
    PackDev* h_packs = nullptr;
    unsigned int* d_bstart = nullptr;
    RungSet* d_rs = nullptr;
    RungSet* h_rs = nullptr;
    BatchStat* d_st = nullptr;
    BatchStat* h_st = nullptr;
    unsigned int total_blocks = 0;
    size_t kappa_smem = 0;
    cudaGraphExec_t gexec = nullptr;
    int gT = 0;
    int chunk = 32;
    int autotune = 0;
    bool tuned = false;
    int long_row = RCP_LONG_ROW;
    bool any_frozen = false;   // some packing holds frozen spheres
    bool any_bounded = false;  // some packing has walls or a container
    std::vector<cudaEvent_t> ev;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    long long launches = 0;
    char err[512] = {0};
};

namespace {

rcp_status bfail(rcp_batch_ctx* b, rcp_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
    return s;
}

#define BK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? RCP_ERR_OOM : RCP_ERR_CUDA, "%s failed: %s", #call, \
                         cudaGetErrorString(e_));                                                  \
    } while (0)

#define BKS(h, expr)                                                   \
    do {                                                               \
        rcp_status s_ = (expr);                                        \
        if (s_ != RCP_OK) return bfail(b, s_, "%s", rcp_last_error(h)); \
    } while (0)

rcp_status batch_refresh(rcp_batch_ctx* b)
{
    for (int p = 0; p < b->B; ++p) b->h_packs[p] = pack_of(b->hs[p]);
    BK(cudaMemcpyAsync(b->d_packs, b->h_packs, sizeof(PackDev) * b->B, cudaMemcpyHostToDevice, b->stream));
    return RCP_OK;
}

// The batched mixed pair kernel for what the batch's packings hold.
decltype(&k_pair_mixed_batch) mixed_batch_kernel(const rcp_batch_ctx* b)
{
    return b->any_bounded ? k_pair_mixed_batch_wl : (b->any_frozen ? k_pair_mixed_batch_fz : k_pair_mixed_batch);
}

void batch_iteration(rcp_batch_ctx* b, int mode)
{
    if (b->precision == RCP_MIXED)
        mixed_batch_kernel(b)<<<b->total_blocks, RCP_PAIR_THREADS, 0, b->stream>>>(b->d_packs, b->d_bstart, b->B, mode);
    else
        k_pair64_batch<<<b->total_blocks, RCP_PAIR_THREADS, 0, b->stream>>>(b->d_packs, b->d_bstart, b->B, mode);
    if (b->precision == RCP_MIXED)
        k_kappa_mixed_batch<<<b->B, 1024, 0, b->stream>>>(b->d_packs, mode);
    else
        k_kappa_step_batch<<<b->B, 1024, b->kappa_smem, b->stream>>>(b->d_packs, mode);
}

rcp_status batch_capture(rcp_batch_ctx* b)
{
    if (b->gexec && b->gT == b->chunk) return RCP_OK;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t graph;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    for (int t = 0; t < b->chunk; ++t) batch_iteration(b, RCP_MODE_ADAM);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return bfail(b, RCP_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, RCP_ERR_CUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    b->gT = b->chunk;
    return RCP_OK;
}

rcp_status batch_status(rcp_batch_ctx* b)
{
    k_batch_status<<<rcp_ceil_div(b->B, 64), 64, 0, b->stream>>>(b->d_packs, b->d_st, b->B);
    BK(cudaPeekAtLastError());
    BK(cudaMemcpyAsync(b->h_st, b->d_st, sizeof(BatchStat) * b->B, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    b->launches += 1;
    for (int p = 0; p < b->B; ++p) {
        RcpCtl* c = b->hs[p]->ctl_h;
        const BatchStat& s = b->h_st[p];
        c->iter = s.iter;
        c->rebuilds = s.rebuilds;
        c->kappa = s.kappa;
        c->E = s.E;
        c->maxdelta = s.maxdelta;
        c->pairs = s.pairs;
        c->halted = s.halted;
        c->stopped = s.stopped;
        c->need_rebuild = s.need_rebuild;
        c->status = s.status;
        c->verify = s.verify;
        c->parity = s.parity;
    }
    return RCP_OK;
}

// Rebuild the flagged packings, phases interleaved across their streams.
rcp_status batch_build(rcp_batch_ctx* b, const std::vector<int>& which)
{
    if (which.empty()) return RCP_OK;
    for (int p : which) BKS(b->hs[p], build_a(b->hs[p]));
    for (int p : which) BK(cudaStreamSynchronize(b->hs[p]->stream));
    for (int p : which) BKS(b->hs[p], build_b(b->hs[p]));
    for (int p : which) BK(cudaStreamSynchronize(b->hs[p]->stream));
    for (int p : which) {
        rcp_ctx* h = b->hs[p];
        BKS(h, build_c(h));
        BK(cudaEventRecord(b->ev[p], h->stream));
        BK(cudaStreamWaitEvent(b->stream, b->ev[p], 0));
        b->launches += 0;
    }
    return batch_refresh(b);
}

// Autotuner: the long-row threshold of the mixed pair kernel, chosen by
// timing the batched kernel in gradient mode (no state change) for each
// candidate; then the graph chunk, chosen by timing replays.
rcp_status batch_autotune_rows(rcp_batch_ctx* b)
{
    if (b->precision != RCP_MIXED) return RCP_OK;
    // thresholds up to 32: a short row keeps its pre-test marks in one
    // 32-bit word (the kernel walks longer rows with a warp)
    const unsigned int cand[3] = {8, 16, 32};
    float best = 1e30f;
    unsigned int pick = RCP_LONG_ROW;
    for (unsigned int lr : cand) {
        for (rcp_ctx* h : b->hs) {
            h->c.long_row = lr;
            BKS(h, relist_long(h));
        }
        for (rcp_ctx* h : b->hs) BK(cudaStreamSynchronize(h->stream));
        BKS(b->hs[0], batch_refresh(b));
        for (int w = 0; w < 2; ++w)
            mixed_batch_kernel(b)<<<b->total_blocks, RCP_PAIR_THREADS, 0, b->stream>>>(b->d_packs, b->d_bstart, b->B,
                                                                                    RCP_MODE_GRAD);
        BK(cudaEventRecord(b->t0, b->stream));
        for (int w = 0; w < 5; ++w)
            mixed_batch_kernel(b)<<<b->total_blocks, RCP_PAIR_THREADS, 0, b->stream>>>(b->d_packs, b->d_bstart, b->B,
                                                                                    RCP_MODE_GRAD);
        BK(cudaEventRecord(b->t1, b->stream));
        BK(cudaEventSynchronize(b->t1));
        float ms = 0.f;
        BK(cudaEventElapsedTime(&ms, b->t0, b->t1));
        b->launches += 7;
        if (ms < best) {
            best = ms;
            pick = lr;
        }
    }
    for (rcp_ctx* h : b->hs) {
        h->c.long_row = pick;
        BKS(h, relist_long(h));
        h->gexec ? (void)cudaGraphExecDestroy(h->gexec) : (void)0;
        h->gexec = nullptr;  // the packing's own graph bakes its constants in
    }
    for (rcp_ctx* h : b->hs) BK(cudaStreamSynchronize(h->stream));
    b->long_row = (int)pick;
    return batch_refresh(b);
}

}  // namespace

extern "C" {

rcp_status rcp_batch_create(rcp_handle* hs, int B, int autotune, rcp_batch* out)
{
    if (!out || !hs || B < 1) return RCP_ERR_ARG;
    *out = nullptr;
    rcp_batch_ctx* b = new rcp_batch_ctx();
    b->B = B;
    b->autotune = autotune;
    b->precision = hs[0] ? hs[0]->cfg.precision : 0;
    rcp_status st = [&]() -> rcp_status {
        int dev0 = hs[0] ? hs[0]->device : 0;
        unsigned int blocks = 0;
        long long maxM = 1;
        std::vector<unsigned int> bstart(B);
        for (int p = 0; p < B; ++p) {
            rcp_ctx* h = hs[p];
            if (!h) return bfail(b, RCP_ERR_ARG, "handle %d is NULL", p);
            if (h->device != dev0) return bfail(b, RCP_ERR_ARG, "handle %d lives on another device", p);
            if (h->cfg.precision != b->precision) return bfail(b, RCP_ERR_ARG, "handles mix precisions");
            for (int q = 0; q < p; ++q)
                if (hs[q] == h) return bfail(b, RCP_ERR_ARG, "handle %d appears twice", p);
            const PackDev q = pack_of(h);
            if (q.nparts > 8192)
                return bfail(b, RCP_ERR_CAPACITY, "packing %d has %u block partials (at most 8192 in a batch)", p,
                             q.nparts);
            long long M = 1;
            while (M < (long long)q.nparts) M <<= 1;
            if (M > maxM) maxM = M;
            bstart[p] = blocks;
            blocks += q.nblocks;
            b->hs.push_back(h);
            if (h->c.nfrozen > 0) b->any_frozen = true;
            if (h->c.bounded) b->any_bounded = true;
            h->stream = h->own_stream;
        }
        b->total_blocks = blocks;
        b->kappa_smem = 2 * sizeof(double) * (size_t)maxM;
        BK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        BK(cudaMalloc(&b->d_packs, sizeof(PackDev) * B));
        BK(cudaMallocHost(&b->h_packs, sizeof(PackDev) * B));
        BK(cudaMalloc(&b->d_bstart, sizeof(unsigned int) * B));
        BK(cudaMalloc(&b->d_rs, sizeof(RungSet) * B));
        BK(cudaMallocHost(&b->h_rs, sizeof(RungSet) * B));
        BK(cudaMalloc(&b->d_st, sizeof(BatchStat) * B));
        BK(cudaMallocHost(&b->h_st, sizeof(BatchStat) * B));
        BK(cudaEventCreate(&b->t0));
        BK(cudaEventCreate(&b->t1));
        b->ev.resize(B);
        for (int p = 0; p < B; ++p) BK(cudaEventCreateWithFlags(&b->ev[p], cudaEventDisableTiming));
        BK(cudaMemcpy(b->d_bstart, bstart.data(), sizeof(unsigned int) * B, cudaMemcpyHostToDevice));
        BK(cudaFuncSetAttribute(k_kappa_step_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 8192 * 8));
        for (rcp_ctx* h : b->hs) BK(cudaStreamSynchronize(h->stream));
        return batch_refresh(b);
    }();
    if (st != RCP_OK) {
        // keep the message for the caller through the first handle
        if (hs[0]) snprintf(hs[0]->err, sizeof(hs[0]->err), "%s", b->err);
        rcp_batch_destroy(b);
        return st;
    }
    *out = b;
    return RCP_OK;
}

rcp_status rcp_batch_destroy(rcp_batch b)
{
    if (!b) return RCP_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->d_packs) cudaFree(b->d_packs);
    if (b->h_packs) cudaFreeHost(b->h_packs);
    if (b->d_bstart) cudaFree(b->d_bstart);
    if (b->d_rs) cudaFree(b->d_rs);
    if (b->h_rs) cudaFreeHost(b->h_rs);
    if (b->d_st) cudaFree(b->d_st);
    if (b->h_st) cudaFreeHost(b->h_st);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return RCP_OK;
}

const char* rcp_batch_last_error(rcp_batch b) { return b ? b->err : ""; }

rcp_status rcp_batch_tuning(rcp_batch b, int* long_row, int* chunk)
{
    if (!b) return RCP_ERR_ARG;
    if (long_row) *long_row = b->long_row;
    if (chunk) *chunk = b->chunk;
    return RCP_OK;
}

rcp_status rcp_batch_run(rcp_batch b, const rcp_stop* stop, rcp_result* outs)
{
    if (!b) return RCP_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    rcp_stop st = {0, 0.0, 1};
    if (stop) st = *stop;
    const long long launches0 = b->launches;
    if (auto s = batch_status(b)) return s;
    std::vector<long long> call_start(b->B);
    std::vector<long long> hl0(b->B);
    for (int p = 0; p < b->B; ++p) {
        call_start[p] = b->hs[p]->ctl_h->iter;
        hl0[p] = b->hs[p]->launches;
    }
    std::vector<rcp_status> result(b->B, RCP_OK);
    std::vector<int> flagged;
    int chunk_phase = b->autotune && !b->tuned ? 0 : -1;  // chunk candidates still to time
    const int chunks[4] = {8, 16, 32, 64};
    float chunk_ms[4] = {0, 0, 0, 0};
    long long chunk_it[4] = {0, 0, 0, 0};
    for (;;) {
        int active = 0;
        flagged.clear();
        bool verified = false;
        for (int p = 0; p < b->B; ++p) {
            rcp_ctx* h = b->hs[p];
            RungSet& rs = b->h_rs[p];
            rs.active = 0;
            if (h->ctl_h->verify) {
                bool s = false;
                if (verify_stop_mixed(h, &s) != RCP_OK) return bfail(b, RCP_ERR_CUDA, "packing %d: %s", p, h->err);
                verified = true;
                continue;
            }
            long long limit = 0;
            int fin = 0;
            const PlanResult pr = plan_replay(h, call_start[p], st.max_iters, &limit, &fin);
            if (pr == PLAN_ERROR) result[p] = (rcp_status)h->ctl_h->status;
            if (pr == PLAN_MAXITER) result[p] = RCP_ERR_MAXITER;
            if (pr != PLAN_RUN) continue;
            rs.mu = h->mu;
            rs.eta_x = h->eta_x;
            rs.eta_k = h->eta_k;
            rs.tol = h->cfg.tol;
            rs.iter_limit = limit;
            rs.final_rung = fin;
            rs.active = 1;
            ++active;
            if (!h->built || h->ctl_h->need_rebuild) flagged.push_back(p);
        }
        if (verified) {
            if (auto s = batch_status(b)) return s;
            continue;
        }
        if (active == 0) break;
        if (st.max_seconds > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >= st.max_seconds)
            break;
        if (auto s = batch_build(b, flagged)) return s;
        if (b->autotune && !b->tuned && chunk_phase == 0) {
            if (auto s = batch_autotune_rows(b)) return s;
        }
        if (chunk_phase >= 0) b->chunk = chunks[chunk_phase];
        if (auto s = batch_capture(b)) return s;
        BK(cudaMemcpyAsync(b->d_rs, b->h_rs, sizeof(RungSet) * b->B, cudaMemcpyHostToDevice, b->stream));
        k_batch_set<<<rcp_ceil_div(b->B, 64), 64, 0, b->stream>>>(b->d_packs, b->d_rs, b->B);
        BK(cudaPeekAtLastError());
        long long it_before = 0;
        for (int p = 0; p < b->B; ++p) it_before += b->hs[p]->ctl_h->iter;
        BK(cudaEventRecord(b->t0, b->stream));
        BK(cudaGraphLaunch(b->gexec, b->stream));
        BK(cudaEventRecord(b->t1, b->stream));
        int per_iter = 2;
        b->launches += 1 + (long long)b->gT * per_iter;
        if (auto s = batch_status(b)) return s;
        if (chunk_phase >= 0) {
            float ms = 0.f;
            BK(cudaEventElapsedTime(&ms, b->t0, b->t1));
            long long it_after = 0;
            for (int p = 0; p < b->B; ++p) it_after += b->hs[p]->ctl_h->iter;
            chunk_ms[chunk_phase] += ms;
            chunk_it[chunk_phase] += it_after - it_before;
            if (chunk_it[chunk_phase] >= 4LL * b->chunk * b->B || chunk_ms[chunk_phase] > 50.f) ++chunk_phase;
            if (chunk_phase == 4) {
                double best = 1e30;
                int pick = 32;
                for (int k = 0; k < 4; ++k)
                    if (chunk_it[k] > 0 && chunk_ms[k] / chunk_it[k] < best) {
                        best = chunk_ms[k] / chunk_it[k];
                        pick = chunks[k];
                    }
                b->chunk = pick;
                b->tuned = true;
                chunk_phase = -1;
            }
        }
    }
    // shrink the packings that reached the criterion
    for (int p = 0; p < b->B; ++p) {
        rcp_ctx* h = b->hs[p];
        if (h->ctl_h->stopped && st.shrink) {
            if (do_shrink(h) != RCP_OK) result[p] = RCP_ERR_CUDA;
        } else {
            if (sync_ctl(h) != RCP_OK) result[p] = RCP_ERR_CUDA;
        }
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rcp_status worst = RCP_OK;
    for (int p = 0; p < b->B; ++p) {
        if (outs) fill_result(b->hs[p], &outs[p], secs, b->hs[p]->launches - hl0[p]);
        if (outs) outs[p].launches = (p == 0) ? b->launches - launches0 : 0;
        if (result[p] != RCP_OK && worst == RCP_OK) worst = result[p];
    }
    if (worst != RCP_OK) bfail(b, worst, "a packing ended with %s", rcp_status_str(worst));
    return worst;
}

}  // extern "C"
