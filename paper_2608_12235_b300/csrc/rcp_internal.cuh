// rcp_internal.cuh -- shared declarations of the CUDA implementation.
//
// The whole library is compiled with -fmad=false so that every binary64
// expression rounds exactly as written (IEEE add, multiply, divide and sqrt
// are correctly rounded on both the GPU and the host); binary32 kernels that
// want fused multiply-adds ask for them with __fmaf_rn.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rcp.h"

#define RCP_KMAX 32
#define RCP_NBITS_AXIS 19
#define RCP_NMAX_AXIS (1u << RCP_NBITS_AXIS)
#define RCP_PAIR_THREADS 256
#define RCP_TREE 1024          // elements per block of a tree-reduction pass
#ifndef RCP_LONG_ROW
#define RCP_LONG_ROW 32        // default: rows longer than this get a warp in the mixed pair kernel (<= 32)
#endif
#ifndef RCP_LONG_BLOCKS_MAX
#define RCP_LONG_BLOCKS_MAX 592  // most blocks (8 warps each) that loop over the long rows
#endif
#ifndef RCP_LONG_DIV
#define RCP_LONG_DIV 1536        // one long-row block per this many spheres (at least 2)
#endif
#define RCP_WARP_ROW_THREADS 128   // binary64 warp-per-row kernel: 4 rows per block
#define RCP_WARP_ROW_MAX_N 4096    // binary64 packings up to this size take a warp per row (measured
                                   // crossover: 2.5x faster at N = 1440, 2.8x slower at N = 2e4)

// Device-resident control block of one packing.  Kernels read the optimiser
// scalars and the current rung's values from here, so one captured graph
// serves every rung and both buffer parities.
// Binary32 scalars of one mixed-precision iteration, derived from the
// binary64 control values by mix_fill whenever those change (three binary64
// divisions: far too slow to repeat in every block of the pair kernel).
struct MixScalars {
    float kappa, kappa_lo, rkappa, eps, rh1, rh2, be1, be2, o1, o2, eta, aeps;
    float limA, limB;  // theta sigma_i (1 - 1e-5) = limA D_i + limB
};
#define RCP_MIX_SRC 6  // binary64 values the scalars derive from: kappa, b1, b2, eta_x, kappa_b, sigma0

struct RcpCtl {
    // written by the host (through k_set_rung) before a replay
    double mu, eta_x, eta_k, tol;
    long long iter_limit;   // halt when iter reaches this
    int final_rung;
    int verify;             // mixed precision: stop candidate awaiting FP64 check
    // optimiser scalars
    double kappa, mk, vk, b1, b2;
    long long iter;
    int parity;             // 0: buffer A holds the current positions
    // flags
    int halted, stopped, need_rebuild, status;
    unsigned int disp_flag;   // some sphere used up its skin budget
    unsigned int kbud_bits;   // binary32 bits of min_i 2 (theta sigma_i - |x_i - x_i^b|) / D_i
    // last evaluation
    double E, dEdk, maxdelta;
    unsigned long long maxdelta_bits;
    // neighbour structure
    double kappa_b, sigma0;
    unsigned long long rho_max_bits;
    unsigned long long rho_lvl_bits[RCP_KMAX];
    unsigned long long lvl_count[RCP_KMAX];
    unsigned long long pair_cursor;   // entries emitted by the pair search
    unsigned int search_heavy;        // search windows queued for k_search_heavy
    double rho_lvl[RCP_KMAX];
    float rho_lvl_f[RCP_KMAX];   // fl32 of rho_lvl (the search windows' binary32 radii)
    int nlev;
    int ng[RCP_KMAX][3];
    unsigned long long cell_off[RCP_KMAX + 1];  // first entry of each class in the dense cell table
    long long rebuilds;
    unsigned long long pairs;
    unsigned int n_long;      // rows longer than RCP_LONG_ROW
    // constants and one-off results
    double SD, SD2, SD3, SD4;   // moments of the mobile spheres' D^0
    double SF2, SF3;            // sums of F^2 and F^3 over the frozen spheres
    unsigned long long shrink_bits;
    unsigned long long md64_bits;
    double kappa_c, phi;
    // binary32 scalars of the next mixed iteration and the values they came from
    MixScalars mix;
    double mix_src[RCP_MIX_SRC];
    // device-side loop of a replayed graph (k_loop_cond)
    long long loop_last_iter;        // iter after the previous body pass of this replay (-1: none yet)
    unsigned long long body_passes;  // body passes run so far (kernel accounting)
};

// Kernel parameters that never change during a run.
struct RcpConst {
    long long N;
    double L[3];
    double halfL[3];
    double V;
    double eps, beta1, beta2, adam_eps;
    double skin_s, skin_theta;
    double Lmin, Lmax;
    double stop_margin;     // 0: binary64 overlaps; > 0: relative band that triggers a binary64 check
    double cell_occ;        // target spheres per cell of a class grid
    float qscale[3];        // qspan_a / 2^32: fixed-point unit of axis a
    float qinv[3];          // 2^32 / qspan_a
    double qspan[3];        // length a record's axis covers: L_a (periodic), 2 L_a (bounded)
    double qoff[3];         // coordinate of q = 0: 0 (periodic), -L_a / 2 (bounded)
    float qo_hi[3], qo_lo[3];  // qoff as an unevaluated binary32 sum
    float Llo[3];           // L_a - Lf[a]
    double invL[3];         // 1 / L_a
    float invLf[3];         // fl32(1 / L_a)
    int pow2L;              // bit a: L_a is a power of two, so x / L_a == x * (1 / L_a) exactly
    float Lf[3];            // L_a in binary32
    float qs_hi[3], qs_lo[3];  // qspan_a 2^-32 as an unevaluated binary32 sum
    float qmargin;             // 2 max_a qscale[a]: absolute margin of the mixed pre-test
    unsigned int canon;        // 1: binary64 path (canonical sums); 0: mixed path
    int dim;                   // the caller's dimension: 3, or 2 (disks held in the plane z = L_z / 2)
    unsigned int long_row;     // rows longer than this get a warp (mixed; binary64 when long64)
    int long64;                // binary64 packing above RCP_WARP_ROW_MAX_N: long rows by k_pair64_long
    unsigned int long_blocks;  // blocks of the mixed pair kernel that serve long rows
    long long nfrozen;         // frozen spheres
    int walls;                 // bit a: flat walls at 0 and L_a bound axis a
    int container;             // curved wall: 0 none, 1 ball (disk when d = 2), 2 cylinder about z
    int caxes;                 // the container's axes (bit a)
    int bounded;               // axes without minimum image or wrap: flat walls and the container's
    double Rc;                 // container radius: min L_a / 2 over its axes (centre L / 2)
    float Rc_hi, Rc_lo;        // Rc as an unevaluated binary32 sum (mixed wall terms)
    float wmargin;             // 2^-20 max_a L_a: absolute margin of the mixed wall pre-test
    double Vs;                 // volume the spheres fill (kappa_0, phi): the container's, else V
};

// Pair record of one sphere: 32-bit fixed-point position q_a = floor(x_a/L_a
// 2^32) (integer subtraction wraps, which is exactly the minimum image), the
// binary32 remainder l_a = x_a/L_a 2^32 - q_a in [0, 1), and D_i^0 as an
// unevaluated binary32 sum.  A bounded axis (flat walls or the container's)
// records (x_a + L_a/2) / (2 L_a) instead, so the plain difference of two
// listed spheres never wraps.  One 32-byte sector per gather; the first 16
// bytes (integer position and fl32(D_i^0)) are all the pre-test reads.
struct __align__(32) MixRec {
    int4 q;    // qx, qy, qz, and the bits of fl32(D_i^0)
    float4 l;  // lx, ly, lz, D_i^0 - fl32(D_i^0)
};
// Everything a pair kernel and the kappa step need about one packing, for
// the batched kernels (one device array entry per packing).
struct PackDev {
    RcpCtl* ctl;
    RcpConst c;
    double4_32a *xA, *xB, *xb;
    double *m64, *v64;
    float *m32, *v32;
    MixRec *rA, *rB, *rb;
    const unsigned int *rowptr, *col, *long_rows;
    double *part_e, *part_k;
    double* g;
    unsigned int nparts;   // partial sums one pair launch writes
    unsigned int nblocks;  // blocks of one pair launch
};

enum { RCP_MODE_ADAM = 0, RCP_MODE_GRAD = 1 };

#define RCP_PI 3.141592653589793

// ---- frozen spheres ----
// A stage of the sequential cascade (Sec. IV) holds the coarser classes
// fixed while a finer class is inflated among them.  A negative D0 = -F marks
// such a frozen sphere: its contact diameter is F whatever kappa is, Adam
// does not move it, and its coordinates carry no gradient.
__device__ __forceinline__ double size_at(double D0, double kappa) { return D0 >= 0.0 ? kappa * D0 : -D0; }
__device__ __forceinline__ double mobile_part(double D0) { return D0 > 0.0 ? D0 : 0.0; }

// ---- binary64 pair pre-test ----
// A listed pair with fl(r^2) > fl(fl(d d) (1 + 1e-12)) cannot overlap in
// binary64: then r^2 > d^2 (1 + 0.9999e-12), so fl(sqrt(r^2)) > d (1 + 4e-13)
// and fl(r / d) > 1, i.e. delta = 1 - r/d <= 0 (each step rounds by at most
// 2^-53 relative).  Such pairs skip the square root and the division, which
// are long sequences on B300's binary64 pipe; every pair that may overlap
// still takes the oracle's exact operations, so results are unchanged.
#define RCP_NO_OVERLAP_MARGIN (1.0 + 1e-12)

// 2Sum accumulation: s + c carries the sum of the added binary32 terms to
// within about one rounding of the result (Knuth's TwoSum; no FMA contraction
// in this library, so the error term is exact).
__device__ __forceinline__ void acc2(float& s, float& c, float x)
{
    const float t = s + x;
    const float z = t - s;
    c = c + ((s - (t - z)) + (x - z));
    s = t;
}

// Warp sum of compensated pairs; the full (s, c) lands in lane 0.
__device__ __forceinline__ void warp_sum2(float& s, float& c)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_down_sync(0xffffffffu, s, o);
        const float co = __shfl_down_sync(0xffffffffu, c, o);
        acc2(s, c, so);
        c = c + co;
    }
}

// ---- small helpers ----
// Binary64 coordinate of a fixed-point record axis: (q + l) qspan 2^-32 +
// qoff; a periodic axis (qoff = 0, qspan = L) wraps into [0, L), a bounded
// one (qspan = 2 L, qoff = -L/2: room on both sides of the walls) does not.
__device__ __forceinline__ double from_fixed(int q, float l, const RcpConst& c, int a)
{
    double v = ((double)(unsigned int)q + (double)l) * (c.qspan[a] * 0x1.0p-32);
    if ((c.bounded >> a) & 1) return v + c.qoff[a];
    if (v >= c.L[a]) v = v - c.L[a];
    return v;
}

#define RCP_KBUD_INF 0x7F800000u
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// The binary32 scalars of an iteration from the control block (binary64).
__device__ __forceinline__ void mix_scalars(const RcpCtl* ctl, const RcpConst& c, MixScalars& s)
{
    const double b1 = ctl->b1 * c.beta1, b2 = ctl->b2 * c.beta2;
    s.kappa = (float)ctl->kappa;
    s.kappa_lo = (float)(ctl->kappa - (double)s.kappa);
    s.rkappa = (float)(1.0 / ctl->kappa);
    s.eps = (float)c.eps;
    s.rh1 = (float)(1.0 / (1.0 - b1));
    s.rh2 = (float)(1.0 / (1.0 - b2));
    s.be1 = (float)c.beta1;
    s.be2 = (float)c.beta2;
    s.o1 = (float)(1.0 - c.beta1);
    s.o2 = (float)(1.0 - c.beta2);
    s.eta = (float)ctl->eta_x;
    s.aeps = (float)c.adam_eps;
    const double mth = c.skin_theta * (1.0 - 1e-5);
    s.limA = (float)(mth * c.skin_s * ctl->kappa_b);
    s.limB = (float)(mth * ctl->sigma0);
}

__device__ __forceinline__ double mix_src_value(const RcpCtl* ctl, int k)
{
    switch (k) {
    case 0: return ctl->kappa;
    case 1: return ctl->b1;
    case 2: return ctl->b2;
    case 3: return ctl->eta_x;
    case 4: return ctl->kappa_b;
    default: return ctl->sigma0;
    }
}

// Store the scalars of the next iteration in the control block (one thread;
// called by every kernel that changes one of the source values).
__device__ __forceinline__ void mix_fill(RcpCtl* ctl, const RcpConst& c)
{
    MixScalars s;
    mix_scalars(ctl, c, s);
    ctl->mix = s;
    for (int k = 0; k < RCP_MIX_SRC; ++k) ctl->mix_src[k] = mix_src_value(ctl, k);
}

static inline unsigned int rcp_ceil_div(unsigned long long a, unsigned long long b) { return (unsigned int)((a + b - 1) / b); }

// ---- kernels (rcp_kernels.cu) ----
__global__ void k_init_positions(unsigned long long seed, long long N, RcpConst c, const double* D0, double4_32a* x);
__global__ void k_tree_terms(const double* D0, long long N, int power, double* out);
__global__ void k_tree_pass(const double* in, long long n, double* out);
__global__ void k_kappa0(RcpCtl* ctl, double phi0, double V, int dim);
__global__ void k_set_rung(RcpCtl* ctl, RcpConst c, double mu, double eta_x, double eta_k, double tol,
                           long long iter_limit, int final_rung);
__global__ void k_clear_halt(RcpCtl* ctl);
__global__ void k_loop_cond(RcpCtl* ctl, cudaGraphConditionalHandle hc);
__global__ void k_set_positions(long long N, RcpConst c, const double* xin, const double* D0, double4_32a* x,
                                const unsigned int* perm, const RcpCtl* ctl = nullptr, double4_32a* xB = nullptr);
__global__ void k_get_positions(long long N, RcpConst c, const double4_32a* x, double* out, const unsigned int* perm);
__global__ void k_place_draw(unsigned long long seed, long long N, long long r, int k, RcpConst c, const double* D0,
                             const int* lvl, const unsigned char* placed, unsigned char* reject, double4_32a* x);
__global__ void k_place_accept(RcpCtl* ctl, long long N, int k, const int* lvl, unsigned char* placed,
                               const unsigned char* reject);
__global__ void k_place_conflicts(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                                  const double* rho, const int* lvl, const unsigned int* idx_sorted, const float4* xsf,
                                  const uint2* cells, const double* D0, const unsigned char* placed,
                                  unsigned char* reject, int kcur);
__global__ void k_perm3(long long N, RcpConst c, const unsigned int* perm, const double* in, double* out,
                        int to_caller);
__global__ void k_pair64(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
                         const unsigned int* rowptr, const unsigned int* col, const double4_32a* xb,
                         double* part_e, double* part_k, int mode, double* g_out, const double* row_e,
                         const double* row_k);
__global__ void k_pair64_long(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
                              const unsigned int* rowptr, const unsigned int* col, const unsigned int* long_rows,
                              const double4_32a* xb, double* row_e, double* row_k, int mode, double* g_out);
__global__ void k_kappa_step(RcpCtl* ctl, RcpConst c, const double* part_e, const double* part_k,
                             long long nb, int mode);
__device__ void kappa_close(RcpCtl* ctl, const RcpConst& c, double se, double sk, int mode);
__global__ void k_kappa_mixed(RcpCtl* ctl, RcpConst c, const double* part_e, const double* part_k, long long n,
                              int mode);
__global__ void k_kappa_mixed_batch(const PackDev* P, int mode);
// Per-packing rung values for a batched replay, and the status read back.
struct RungSet {
    double mu, eta_x, eta_k, tol;
    long long iter_limit;
    int final_rung;
    int active;   // 0: the packing sits this replay out
};
struct BatchStat {
    long long iter, rebuilds;
    double kappa, E, maxdelta;
    unsigned long long pairs;
    int halted, stopped, need_rebuild, status, verify, parity;
};
__global__ void k_batch_set(const PackDev* P, const RungSet* rs, int B);
__global__ void k_batch_status(const PackDev* P, BatchStat* out, int B);
__global__ void k_pair64_batch(const PackDev* P, const unsigned int* bstart, int B, int mode);
__global__ void k_pair64_warp(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
                              const unsigned int* rowptr, const unsigned int* col, const double4_32a* xb,
                              double* row_e, double* row_k, int mode, double* g_out);
__global__ void k_kappa_step_batch(const PackDev* P, int mode);
__global__ void k_pair_mixed_batch(const PackDev* P, const unsigned int* bstart, int B, int mode);
__global__ void k_pair_mixed_batch_fz(const PackDev* P, const unsigned int* bstart, int B, int mode);
__global__ void k_pair_mixed_batch_wl(const PackDev* P, const unsigned int* bstart, int B, int mode);
__global__ void k_tree_pass2(const double* ina, const double* inb, long long n, double* outa, double* outb);
__global__ void k_adam64(RcpCtl* ctl, RcpConst c, double4_32a* xA, double4_32a* xB, double* m, double* v,
                         const double* g, const double4_32a* xb, double eta_x);
__global__ void k_adam_kappa(RcpCtl* ctl, RcpConst c, double dEdk, double eta_k);
__global__ void k_disp_check(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const double4_32a* xb);
__global__ void k_shrink(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                         const unsigned int* rowptr, const unsigned int* col);
__global__ void k_shrink_final(RcpCtl* ctl, RcpConst c);

// ---- mixed precision (rcp_mixed.cu) ----
__global__ void k_to_fixed(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                           MixRec* rA, MixRec* rB, MixRec* rb);
__global__ void k_pair_mixed(RcpCtl* ctl, RcpConst c, float* m, float* v, MixRec* rA, MixRec* rB,
                             const unsigned int* rowptr, const unsigned int* col, const unsigned int* long_rows,
                             const MixRec* rb, double* part_e, double* part_k, int mode, double* g_out);
__global__ void k_pair_mixed_fz(RcpCtl* ctl, RcpConst c, float* m, float* v, MixRec* rA, MixRec* rB,
                                const unsigned int* rowptr, const unsigned int* col, const unsigned int* long_rows,
                                const MixRec* rb, double* part_e, double* part_k, int mode, double* g_out);
__global__ void k_pair_mixed_wl(RcpCtl* ctl, RcpConst c, float* m, float* v, MixRec* rA, MixRec* rB,
                                const unsigned int* rowptr, const unsigned int* col, const unsigned int* long_rows,
                                const MixRec* rb, double* part_e, double* part_k, int mode, double* g_out);
// in rcp_kernels.cu, beside the binary64 wall terms
__global__ void k_maxdelta64(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                             const unsigned int* rowptr, const unsigned int* col);
__global__ void k_verify_final(RcpCtl* ctl, RcpConst c);
__global__ void k_adam_mixed(RcpCtl* ctl, RcpConst c, MixRec* rA, MixRec* rB, float* m, float* v, const double* g,
                             const MixRec* rb, double eta_x);
__global__ void k_mix_refresh(RcpCtl* ctl, RcpConst c);
__global__ void k_from_fixed(RcpCtl* ctl, RcpConst c, const MixRec* rA, const MixRec* rB, const double* D0,
                             double4_32a* xA, double4_32a* xB);
__global__ void k_snap_records(RcpCtl* ctl, long long N, const MixRec* rA, const MixRec* rB, MixRec* rb);

// ---- neighbour structure (rcp_build.cu) ----
__global__ void k_build_begin(RcpCtl* ctl, double sigma0);
__global__ void k_rho(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, double* rho,
                      float4* xf);
__global__ void k_gather_sorted(long long N, const unsigned int* idx_sorted, const float4* xf, float4* xsf);
__global__ void k_level(RcpCtl* ctl, long long N, const double* rho, int* lvl);
__global__ void k_grid(RcpCtl* ctl, RcpConst c);
__global__ void k_cell_key(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const int* lvl,
                           unsigned long long* key);
__global__ void k_cell_pairs(const RcpCtl* ctl, long long N, const unsigned long long* key, int nbits,
                             unsigned long long* ck);
__global__ void k_cell_table(const unsigned int* cptr, unsigned long long ncells, uint2* cells);
__global__ void k_gather_keys(long long N, const unsigned int* sorted, const unsigned long long* key,
                              unsigned long long* skeys);
__global__ void k_scan_block(const unsigned int* in, long long n, unsigned int* out, unsigned int* totals);
__global__ void k_scan_add(unsigned int* out, long long n, const unsigned int* offs);
__global__ void k_permute_state(const RcpCtl* ctl, long long N, const unsigned int* sorted, MixRec* rA, MixRec* rB,
                                double4_32a* xA, double4_32a* xB, const float* m, const float* v, float* m2,
                                float* v2, const double* D0, double* D02, const double* rho, double* rho2,
                                const int* lvl, int* lvl2, const unsigned int* perm, unsigned int* perm2);
__global__ void k_flip_parity(RcpCtl* ctl);
__global__ void k_iota(long long N, unsigned int* out);
__global__ void k_search(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, const MixRec* rA,
                         const MixRec* rB, const double* rho, const int* lvl, const unsigned int* idx_sorted,
                         const float4* xsf, const uint2* cells, unsigned long long* pairs, unsigned long long cap,
                         int nbits, uint2* heavy, unsigned int heavy_cap);
__global__ void k_search_heavy(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB,
                               const MixRec* rA, const MixRec* rB, const double* rho, const int* lvl,
                               const unsigned int* idx_sorted, const float4* xsf, const uint2* cells,
                               unsigned long long* pairs, unsigned long long cap, int nbits, const uint2* heavy,
                               unsigned int heavy_cap);
__global__ void k_rho_mixed(RcpCtl* ctl, RcpConst c, const MixRec* rA, const MixRec* rB, const double* D0,
                            double* rho, float4* xf);
__global__ void k_cell_key_mixed(RcpCtl* ctl, RcpConst c, const MixRec* rA, const MixRec* rB, const int* lvl,
                                 unsigned long long* key);
__global__ void k_row_count(const unsigned long long* pairs, long long P, int nbits, unsigned int* cnt);
__global__ void k_row_scatter(const unsigned long long* pairs, long long P, int nbits, const unsigned int* rowptr,
                              unsigned int* fill, unsigned int* colu);
__global__ void k_row_sort(const unsigned int* rowptr, long long N, const unsigned int* colu, unsigned int* col);
#define RCP_RS_CAP 2048      // row starts per block of k_row_sort
#define RCP_RS_BUF 6144      // entries a block of k_row_sort stages in shared memory (24 KB; a block whose
                             // rows span more sorts them in place in global memory)
__global__ void k_long_flags(const unsigned int* rowptr, long long N, unsigned int long_row, unsigned int* flags);
__global__ void k_long_compact(RcpCtl* ctl, const unsigned int* flags, const unsigned int* offs, long long N,
                               unsigned int* long_rows);
__global__ void k_build_end(RcpCtl* ctl, RcpConst c, const double4_32a* xA, const double4_32a* xB, double4_32a* xb,
                            unsigned long long P);
