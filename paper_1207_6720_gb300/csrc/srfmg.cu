// srfmg.cu -- host side of the FMG-FAS-SR solver: parameter checks, device
// workspace, the level schedule of one FMG cycle (Fig. 2 with the SR steps of
// Fig. 3), CUDA-graph capture and replay, and the C ABI declared in srfmg.h.
#include "srfmg.h"
#include "srfmg_kernels.cuh"
#include "srfmg_fixed.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>   // tracing ranges (no-ops unless a profiler is attached)

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace srfmg;

namespace {

constexpr int kMaxTailLevel = 12;      // levels <= 12 fit one block's shared memory in FP64
constexpr int kTailThreads = kTailBlock;
constexpr int kRhsThreads = 256;
constexpr int kRhsDepth = 12;          // levels reduced per rhs-hierarchy launch
constexpr int kTileMax = 2048;

thread_local std::string g_create_error = "no error";

enum OpKind { OP_RHS, OP_TAIL, OP_DOWN_PI, OP_DOWN, OP_UP, OP_SR_PRE, OP_SEAM, OP_SR_POST, OP_SCALE, OP_DOWN_CHAIN,
              OP_UP_CHAIN };

// Pointers that are only known at solve time are patched through these tags.
enum PtrTag { TAG_NONE = 0, TAG_F = 1, TAG_U = 2 };   // f, u: the caller's pointers of a solve

struct Op {
    OpKind kind;
    int level;
    dim3 grid, block;
    size_t smem;
    RhsArgs rhs;
    LevelArgs lev;
    SegArgs seg;
    TailArgs tail;
    int nseg;
    // tags for pointer fields patched per solve
    PtrTag rhs_in, lev_g, lev_out, tail_g, tail_out, seg_f, seg_u;
    PtrTag seg_uin;   // a V-cycle's pre-leg from the caller's current fine solution
    PtrTag lev_uin;   // a V-cycle's down pass on the finest level of a plan without SR, from u
    // operator of the FP64 kernels (kOpLaplace, kOpVarcoef, kOpBratu; kOpBratuMx: the
    // mixed precision of the Bratu problem, FP32 correction recurrences)
    int opk;
    // fixed-point variant (precision SRFMG_MIXED of -u'' = f and -(a u')' = f): the
    // same op with integer kernels; vc: their variable-coefficient instantiation
    bool fixed, vc;
    fx::RhsArgs frhs;
    fx::LevelArgs flev;
    fx::SegArgs fseg;
    fx::TailArgs ftail;
    fx::ChainArgs fchain;      // OP_DOWN_CHAIN, OP_UP_CHAIN (fixed point only)
    fx::Scale *scale;
    int *status;      // OP_SCALE: the plan's status word
};

// The caller's pointers of one solve, patched into the tagged op fields.
struct Io {
    const double *f;
    double *u;                 // the solution (NULL: not written; functionals only)
    const double *u_ref;       // reference of the functionals, or NULL
    double *fout;              // functionals, kNumFunc per problem, or NULL
    double *fpart;             // the plan's segment partials when fout is set
};

}  // namespace

struct srfmg_plan {
    srfmg_params p;
    int device;
    int M, M0, Mc, nRS, W, b;
    int batch;                     // independent problems solved together (>= 1)
    size_t n;                      // cells per problem
    std::vector<void *> allocs;
    double *ulev[32][2] = {};
    double *glev[32] = {};
    double *seam = nullptr;
    double *uold = nullptr, *uhat = nullptr, *edge = nullptr;   // post-leg option FAS recompute
    double *Ainv = nullptr;
    double *coef[32] = {};         // variable coefficient: face coefficients of levels M0..M
    fx::u64 *fA[32] = {};          // fixed-point variable coefficient: A per face, levels M0..M
    fx::u64 *fBM[32] = {};         // fixed-point variable coefficient: two multiplier words per cell
    int *coef_bad = nullptr;       // variable coefficient: set by the coefficient kernel's check
    fx::Scale *scale = nullptr;    // fixed-point scales (precision SRFMG_MIXED)
    double *fpart = nullptr;       // SR plans: functional partials, kNumFunc per segment and problem
    int *status = nullptr;         // device status word (kStatusNonFinite), read by srfmg_check
    bool solved = false;           // a solve has been enqueued (its coarse solution is kept)
    bool fixed = false;
    double *f_stage = nullptr, *u_stage = nullptr;
    // pipelined host solves (srfmg_solve_host_async): two staging pairs used in
    // turn, copy-in and copy-out streams, and the events that order them
    double *hf[2] = {}, *hu[2] = {};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_join = nullptr, ev_in[2] = {}, ev_solved[2] = {}, ev_out[2] = {};
    int hslot = 0;
    size_t ws_bytes = 0;
    std::vector<Op> ops;
    std::vector<std::string> names;
    cudaStream_t cap_stream = nullptr;
    // captured launch sequences, one per (f, u, u_ref, functionals) pointer set
    // (a solve and an adjoint solve on other buffers keep their own); least
    // recently used out
    static constexpr int kGraphSlots = 4;
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const double *f = nullptr;
        double *u = nullptr;
        const double *u_ref = nullptr;
        double *fout = nullptr;
        unsigned long long used = 0;
    } graphs[kGraphSlots];
    unsigned long long graph_clock = 0;
    bool use_graph = true;
    std::string err = "no error";
};

namespace {

srfmg_status fail(srfmg_plan *h, srfmg_status st, const std::string &msg) {
    if (h) h->err = msg; else g_create_error = msg;
    return st;
}

srfmg_status cuda_fail(srfmg_plan *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, SRFMG_ECUDA, m);
}

bool pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

std::string check_params(const srfmg_params *p) {
    if (!p) return "params is NULL";
    if (p->tail_level != 0 && (p->tail_level < p->log2_n_coarsest || p->tail_level > 12))
        return "tail_level must be 0 or in [log2_n_coarsest, 12]";
    if (p->tile_cells != 0 && (!pow2(p->tile_cells) || p->tile_cells < 64 || p->tile_cells > 2048))
        return "tile_cells must be 0 or a power of two in [64, 2048]";
    if (p->chain_down < 0 || p->chain_down > fx::kChainMax || p->chain_up < 0 || p->chain_up > fx::kChainMax)
        return "chain_down and chain_up must be in [0, 4]";
    if ((p->chain_down >= 2 || p->chain_up >= 2) && (p->precision != SRFMG_MIXED || p->op != SRFMG_OP_LAPLACE))
        return "chain_down and chain_up apply to SRFMG_MIXED with SRFMG_OP_LAPLACE";
    if (p->post_leg != SRFMG_POST_FULL_UPDATE && p->post_leg != SRFMG_POST_FAS_RECOMPUTE)
        return "post_leg must be SRFMG_POST_FULL_UPDATE or SRFMG_POST_FAS_RECOMPUTE";
    if (p->post_leg == SRFMG_POST_FAS_RECOMPUTE &&
        (p->n_sr_levels != 1 || p->tau_edge != SRFMG_TAU_ASSEMBLED || p->n_vcycles != 0 ||
         p->buffer_width >= p->segment_width))
        return "SRFMG_POST_FAS_RECOMPUTE needs n_sr_levels = 1, tau_edge = SRFMG_TAU_ASSEMBLED, n_vcycles = 0 "
               "and buffer_width < segment_width";
    if (p->n_vcycles < 0 || p->n_vcycles > 16) return "n_vcycles must be in [0, 16]";
    if (p->tau_edge != SRFMG_TAU_ASSEMBLED && p->tau_edge != SRFMG_TAU_SEGMENT)
        return "tau_edge must be SRFMG_TAU_ASSEMBLED or SRFMG_TAU_SEGMENT";
    if (p->tau_edge != SRFMG_TAU_ASSEMBLED && p->n_sr_levels == 0) return "tau_edge applies to SR levels only";
    if (p->batch < 0 || p->batch > 65535) return "batch must be in [0, 65535] (0 means 1)";
    if (p->op != SRFMG_OP_LAPLACE && p->op != SRFMG_OP_BRATU && p->op != SRFMG_OP_VARCOEF)
        return "op must be SRFMG_OP_LAPLACE, SRFMG_OP_VARCOEF or SRFMG_OP_BRATU";
    if (p->op != SRFMG_OP_BRATU && p->lambda != 0.0) return "lambda must be 0 unless op is SRFMG_OP_BRATU";
    if (p->op == SRFMG_OP_BRATU && !(p->lambda >= 0.0 && p->lambda <= 1e300))
        return "lambda must be finite and >= 0";
    if (p->precision != SRFMG_FP64 && p->precision != SRFMG_MIXED) return "unknown precision";
    if (p->smoother != SRFMG_SMOOTH_LEX) return "smoother must be SRFMG_SMOOTH_LEX";
    if (p->log2_n_coarsest < 2 || p->log2_n_coarsest > 6) return "log2_n_coarsest must be in [2, 6]";
    if (p->log2_n <= p->log2_n_coarsest || p->log2_n > 28) return "log2_n must be in (log2_n_coarsest, 28]";
    if (p->n_sr_levels < 0 || p->n_sr_levels > 2) return "n_sr_levels must be 0, 1 or 2";
    if (p->n_sr_levels == 2 && p->log2_n < p->log2_n_coarsest + 2)
        return "two SR levels need log2_n >= log2_n_coarsest + 2 (a stored level below them)";
    if (p->nu1 < 1 || p->nu1 > 4 || p->nu2 < 1 || p->nu2 > 4) return "nu1 and nu2 must be in [1, 4]";
    if (p->n_sr_levels >= 1) {
        long long N = 1LL << p->log2_n;
        if (!pow2(p->segment_width) || p->segment_width < 16 || p->segment_width > 4096 ||
            p->segment_width > N)
            return "segment_width must be a power of two in [16, min(4096, N)]";
        // the deepest SR level's segments are segment_width >> (n_sr_levels - 1) cells
        const int wmin = p->segment_width >> (p->n_sr_levels - 1);
        if (p->buffer_width < 2 || p->buffer_width > 64 || (p->buffer_width & 1) || p->buffer_width > wmin)
            return "buffer_width must be even, in [2, 64] and <= the segment width of every SR level";
    }
    return "";
}

// The table of the mixed precision's exponential (exp_mx): 2^(j/256) for
// j < 256, each rounded once from long double, then ln2/256 as a leading double
// and the rest; uploaded to the current device.
cudaError_t upload_exp_table() {
    double tab[258];
    for (int j = 0; j < 256; ++j) tab[j] = (double)exp2l((long double)j / 256.0L);
    const long double L = logl(2.0L) / 256.0L;
    tab[256] = (double)L;
    tab[257] = (double)(L - (long double)tab[256]);
    return cudaMemcpyToSymbol(g_exp2_tab, tab, sizeof(tab));
}

// exp_mx against exp at n evenly spaced points of [lo, hi]: the largest
// relative difference, as the bits of a non-negative double (they order like
// the values) combined by atomicMax.
__global__ void exp_error_kernel(double lo, double hi, int n, unsigned long long *out) {
    unsigned long long worst = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = (n > 1) ? lo + (hi - lo) * ((double)i / (double)(n - 1)) : lo;
        const double ref = exp(x);
        const double d = fabs(exp_mx(x) - ref) / ref;
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        worst = b > worst ? b : worst;
    }
    atomicMax(out, worst);
}

// Inverse of the scaled coarsest operator h^2 L (tridiag(-1,2,-1), 3 in the
// wall rows) by Gauss-Jordan elimination in long double.
std::vector<double> coarsest_inverse(int n) {
    std::vector<long double> A(n * 2 * n, 0.0L);
    auto at = [&](int i, int j) -> long double & { return A[i * 2 * n + j]; };
    for (int i = 0; i < n; ++i) {
        at(i, i) = (i == 0 || i == n - 1) ? 3.0L : 2.0L;
        if (i > 0) at(i, i - 1) = -1.0L;
        if (i < n - 1) at(i, i + 1) = -1.0L;
        at(i, n + i) = 1.0L;
    }
    for (int c = 0; c < n; ++c) {
        long double piv = at(c, c);
        for (int j = 0; j < 2 * n; ++j) at(c, j) /= piv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            long double f = at(r, c);
            if (f == 0.0L) continue;
            for (int j = 0; j < 2 * n; ++j) at(r, j) -= f * at(c, j);
        }
    }
    std::vector<double> inv(n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = (double)at(i, n + j);
    return inv;
}

// Shared-memory layout of a block that sweeps up to `cells` cells: two level
// buffers (solution, right-hand side), the coarse cells it reads, the
// per-chunk carries and (fixed point) the restricted right-hand side of its
// coarse cells; one thread per sweep chunk (rounded up to whole warps), which
// the sweeps require.
size_t sweep_layout(int cells, int *maxlen, int *maxc, int *maxch, int *threads) {
    *maxlen = cells + 2;
    *maxc = cells / 2 + 8;
    *maxch = (cells + kChunk - 1) / kChunk + 2;
    *threads = ((*maxch + 31) / 32) * 32;
    return (size_t)2 * *maxlen + 2 * *maxc + *maxch;
}

size_t tail_smem_doubles(int M0, int Mc) {
    size_t tot = (1u << (Mc + 1)) - (1u << M0);
    return 2 * tot + (1u << Mc) + 8 + 2 * kTailThreads;
}

srfmg_status alloc_dev(srfmg_plan *h, double **out, size_t count) {
    void *ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, SRFMG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(ptr);
    h->ws_bytes += count * sizeof(double);
    *out = (double *)ptr;
    return SRFMG_OK;
}

Op make_op(OpKind k) {
    Op o;
    std::memset(&o, 0, sizeof(o));
    o.kind = k;
    return o;
}

double op_lambda(const srfmg_plan *h) { return h->p.op == SRFMG_OP_BRATU ? h->p.lambda : 0.0; }

// Level pass of a stored level (global smoothing), tile decomposition.
Op level_op(srfmg_plan *h, OpKind kind, int l, const double *u_src, const double *uc_src,
            double *u_out, double *uc_out, double *gc_out) {
    Op o = make_op(kind);
    o.level = l;
    const int n = 1 << l;
    const int nu = (kind == OP_UP) ? h->p.nu2 : h->p.nu1;
    // a level of at most 2^18 cells over the whole batch is latency-bound (a few
    // microseconds per pass whatever its size): smaller tiles spread it over more
    // SMs (measured: 1.8% off the N = 2^24 solve; 128-cell tiles, or 256 up to
    // level 20, were slower); a larger one is throughput-bound, and there the
    // halos of small tiles cost (the batch of 8192 problems: 304 -> 394 ms)
    const bool latency_bound = ((long long)n * h->batch) <= (1LL << 18);
    const int Tmax = latency_bound ? (h->p.tile_cells ? h->p.tile_cells : 256) : kTileMax;
    const int T = n < Tmax ? n : Tmax;
    // halo: each sweep's values become tile-independent (J+2)*kChunk cells
    // after its range start (9 * 9 = 81 cells, J+1 = ceil(72/9); 12 * 9 = 108
    // for the variable coefficient's 11 carry chunks), every sweep shrinks its
    // range by one cell, and the tau stencil reaches 2 cells past the tile
    const int H = 112 * nu;
    o.lev.l = l;
    o.lev.n = n;
    o.lev.tile = T;
    o.lev.halo = H;
    o.lev.nu = nu;
    o.lev.u_src = u_src;
    o.lev.uc_src = uc_src;
    o.lev.u_out = u_out;
    o.lev.uc_out = uc_out;
    o.lev.gc_out = gc_out;
    o.lev.lam = op_lambda(h);
    o.lev.coef = h->coef[l];
    if (l == h->M) {               // finest level without SR: rhs from f
        o.lev.g = nullptr;
        o.lev_g = TAG_F;
        o.lev.g_exp = -2 * l;
    } else {
        o.lev.g = h->glev[l];
        o.lev.g_exp = 0;
    }
    int threads;
    o.grid = dim3(n / T);
    o.smem = sweep_layout(T + 2 * H, &o.lev.maxlen, &o.lev.maxc, &o.lev.maxch, &threads) * sizeof(double);
    o.block = dim3(threads);
    return o;
}

// A segment pass on the SR level L (segments of W >> (M - L) cells with b
// buffer cells).  On the finest level the rhs is f and the post-leg writes the
// caller's u; below it the rhs is the stored g_in = glev[L] and the post-leg
// writes the level array u_out.  u_in: the assembled iterate of a down-leg
// pre-pass (no FMG interpolation).
Op seg_op(srfmg_plan *h, OpKind kind, int L, const double *uc_src, double *uc_out, double *gc_out,
          const double *g_in, const double *u_in, double *u_out) {
    Op o = make_op(kind);
    const int W = h->W >> (h->M - L);
    o.level = L;
    o.seg.M = L;
    o.seg.n = 1 << L;
    o.seg.W = W;
    o.seg.b = h->b;
    o.seg.nu = (kind == OP_SR_POST) ? h->p.nu2 : h->p.nu1;
    o.seg.uc_src = uc_src;
    o.seg.uc_out = uc_out;
    o.seg.gc_out = gc_out;
    o.seg.g_in = g_in;
    o.seg.u_in = u_in;
    o.seg.u_out = u_out;
    o.seg.seam = h->seam;
    o.seg.lam = op_lambda(h);
    o.seg.coef = h->coef[L];
    o.seg.local_tau = (h->p.tau_edge == SRFMG_TAU_SEGMENT);
    if (L == h->M) {
        o.seg_f = TAG_F;
        if (kind == OP_SR_POST) o.seg_u = TAG_U;
    }
    o.nseg = (int)(h->n / h->W);
    if (kind == OP_SEAM) {
        o.grid = dim3((o.nseg + 127) / 128);
        o.block = dim3(128);
        o.smem = 0;
    } else {
        int threads;
        o.grid = dim3(o.nseg);
        o.smem = sweep_layout(W + 2 * h->b, &o.seg.maxlen, &o.seg.maxc, &o.seg.maxch, &threads) * sizeof(double);
        o.block = dim3(threads);
    }
    return o;
}

Op tail_op(srfmg_plan *h, int mode, const double *u_in, const double *g_in, int g_exp,
           double *u_out, bool g_from_f, bool out_is_u) {
    Op o = make_op(OP_TAIL);
    o.level = h->Mc;
    o.tail.M0 = h->M0;
    o.tail.Mc = h->Mc;
    o.tail.nu1 = h->p.nu1;
    o.tail.nu2 = h->p.nu2;
    o.tail.mode = mode;
    o.tail.u_in = u_in;
    o.tail.g_in = g_in;
    o.tail.g_exp = g_exp;
    o.tail.status = h->status;
    o.tail.u_out = u_out;
    o.tail.Ainv = h->Ainv;
    o.tail.lam = op_lambda(h);
    for (int l = 0; l < 32; ++l) o.tail.coef[l] = h->coef[l];
    if (g_from_f) o.tail_g = TAG_F;
    if (out_is_u) o.tail_out = TAG_U;
    o.grid = dim3(1);
    o.block = dim3(kTailThreads);
    o.smem = tail_smem_doubles(h->M0, h->Mc) * sizeof(double);
    return o;
}

// A stored level whose passes may be chained: fixed point, -u'' = f, at most
// 2^18 cells over the whole batch (the latency-bound ones).
bool chainable(const srfmg_plan *h, int l) {
    return h->fixed && h->p.op == SRFMG_OP_LAPLACE && ((long long)1 << l) * h->batch <= (1LL << 18);
}

// A chain of k stored-level passes (fixed point): down from level l (levels l
// .. l-k+1) or up from level l (levels l .. l+k-1); the pointers are set by
// the caller.  Shared memory: U and G of each chain level's held range, the
// coarse cells of an up step, the chunk carries (see the kernels).
Op chain_op(srfmg_plan *h, OpKind kind, int l, int k) {
    Op o = make_op(kind);
    fx::ChainArgs &c = o.fchain;
    const bool down = (kind == OP_DOWN_CHAIN);
    const int fine = down ? l : l + k - 1;     // the chain's finest level
    const int n = 1 << fine;
    const int Tmax = h->p.tile_cells ? h->p.tile_cells : 256;
    const int T = n < Tmax ? n : Tmax;
    const int nu = down ? h->p.nu1 : h->p.nu2;
    o.level = l;
    c.k = k;
    c.l = l;
    c.tile = T;
    c.H = 112 * nu;                            // the halo of level_op
    c.nu = nu;
    c.sc = h->scale;
    int len[fx::kChainMax];
    if (down) {
        int hh = c.H;
        for (int i = k - 1; i >= 0; --i) {
            len[i] = (T >> i) + 2 * hh;
            hh = 2 * hh + c.H;
        }
    } else {
        len[k - 1] = T + 2 * c.H;
        for (int i = k - 2; i >= 0; --i) len[i] = (len[i + 1] >> 1) + 6 + 2 * c.H;
    }
    size_t off = 0;
    int maxlen = 0;
    for (int i = 0; i < k; ++i) {
        c.off[i] = (int)off;
        c.len[i] = len[i];
        off += 2 * (size_t)len[i];
        maxlen = std::max(maxlen, len[i]);
    }
    c.off_c = (int)off;
    if (!down) off += (size_t)maxlen / 2 + 8;
    c.off_x = (int)off;
    const int maxch = (maxlen + kChunk - 1) / kChunk + 2;
    off += (size_t)maxch;
    o.smem = off * sizeof(fx::i64);
    o.grid = dim3(n / T);
    o.block = dim3(((maxch + 31) / 32) * 32);
    o.fixed = true;
    return o;
}

// Fixed-point form of an op (same schedule, same buffers: a level array holds
// doubles or 64-bit integers of the same size).
void to_fixed(srfmg_plan *h, Op &o) {
    o.fixed = true;
    o.vc = (h->p.op == SRFMG_OP_VARCOEF);
    o.scale = h->scale;
    typedef fx::i64 i64;
    switch (o.kind) {
    case OP_RHS:
        o.frhs.sc = h->scale;
        o.frhs.from_f = (o.rhs_in == TAG_F);
        o.frhs.in = (const i64 *)o.rhs.in;
        o.frhs.lin = o.rhs.lin;
        o.frhs.lstop = o.rhs.lstop;
        o.frhs.depth = o.rhs.depth;
        o.frhs.chunk_log = o.rhs.chunk_log;
        for (int l = 0; l < 32; ++l) o.frhs.out[l] = (i64 *)o.rhs.out[l];
        break;
    case OP_DOWN_PI: case OP_DOWN: case OP_UP:
        o.flev.l = o.lev.l; o.flev.n = o.lev.n; o.flev.tile = o.lev.tile; o.flev.halo = o.lev.halo;
        o.flev.nu = o.lev.nu; o.flev.maxlen = o.lev.maxlen; o.flev.maxc = o.lev.maxc; o.flev.maxch = o.lev.maxch;
        o.flev.sc = h->scale;
        o.flev.u_src = (const i64 *)o.lev.u_src;
        o.flev.g = (o.lev_g == TAG_F) ? nullptr : (const i64 *)o.lev.g;
        o.flev.uc_src = (const i64 *)o.lev.uc_src;
        o.flev.u_out = (i64 *)o.lev.u_out;
        o.flev.uc_out = (i64 *)o.lev.uc_out;
        o.flev.gc_out = (i64 *)o.lev.gc_out;
        o.flev.cA = h->fA[o.lev.l];
        o.flev.cBM = h->fBM[o.lev.l];
        break;
    case OP_SR_PRE: case OP_SEAM: case OP_SR_POST:
        o.fseg.M = o.seg.M; o.fseg.n = o.seg.n; o.fseg.W = o.seg.W; o.fseg.b = o.seg.b; o.fseg.nu = o.seg.nu;
        o.fseg.maxlen = o.seg.maxlen; o.fseg.maxc = o.seg.maxc; o.fseg.maxch = o.seg.maxch;
        o.fseg.sc = h->scale;
        o.fseg.uc_src = (const i64 *)o.seg.uc_src;
        o.fseg.uc_out = (i64 *)o.seg.uc_out;
        o.fseg.gc_out = (i64 *)o.seg.gc_out;
        o.fseg.seam = (i64 *)o.seg.seam;
        o.fseg.g_in = (const i64 *)o.seg.g_in;
        o.fseg.u_in = (const i64 *)o.seg.u_in;
        o.fseg.u_out_fx = (i64 *)o.seg.u_out;   // a level below the finest (the finest: patched per solve)
        o.fseg.local_tau = o.seg.local_tau;
        o.fseg.cA = h->fA[o.seg.M];
        o.fseg.cBM = h->fBM[o.seg.M];
        o.fseg.u_old_out = (i64 *)o.seg.u_old_out;
        o.fseg.edge_out = (i64 *)o.seg.edge_out;
        o.fseg.uc_corr = (const i64 *)o.seg.uc_corr;
        o.fseg.uhat = (const i64 *)o.seg.uhat;
        o.fseg.edge_in = (const i64 *)o.seg.edge_in;
        o.fseg.nu_pre = o.seg.nu_pre;
        break;
    case OP_TAIL:
        o.ftail.M0 = o.tail.M0; o.ftail.Mc = o.tail.Mc; o.ftail.nu1 = o.tail.nu1; o.ftail.nu2 = o.tail.nu2;
        o.ftail.mode = o.tail.mode;
        o.ftail.sc = h->scale;
        o.ftail.u_in = (const i64 *)o.tail.u_in;
        o.ftail.g_in = (o.tail_g == TAG_F) ? nullptr : (const i64 *)o.tail.g_in;
        o.ftail.u_out = (i64 *)o.tail.u_out;
        o.ftail.Ainv = o.tail.Ainv;
        for (int l = 0; l < 32; ++l) {
            o.ftail.cA[l] = h->fA[l];
            o.ftail.cBM[l] = h->fBM[l];
        }
        o.ftail.coef0 = h->coef[h->M0];
        break;
    case OP_SCALE: case OP_DOWN_CHAIN: case OP_UP_CHAIN:
        break;
    }
}

// The level schedule of one FMG cycle.  cur[l] tracks which of the two
// buffers of level l holds its current iterate.
void build_schedule_ops(srfmg_plan *h) {
    const int M = h->M, Mc = h->Mc;
    int cur[32] = {0};
    auto U = [&](int l) { return h->ulev[l][cur[l]]; };
    auto Unext = [&](int l) { return h->ulev[l][cur[l] ^ 1]; };

    // K1: rhs hierarchy g_{M-1} .. g_Mc from f
    if (Mc < M) {
        int lin = M;
        while (lin > Mc) {
            int depth = lin - Mc < kRhsDepth ? lin - Mc : kRhsDepth;
            Op o = make_op(OP_RHS);
            o.level = lin;
            o.rhs.lin = lin;
            o.rhs.lstop = lin - depth;
            o.rhs.depth = depth;
            // at least 4096 cells per block: a shallow reduction (few levels
            // above the tail) would otherwise launch one tiny block per 2^depth cells
            o.rhs.chunk_log = std::max(depth, std::min(lin, 12));
            if (lin == M) { o.rhs_in = TAG_F; o.rhs.in_exp = -2 * M; o.rhs.status = h->status; }
            else { o.rhs.in = h->glev[lin]; o.rhs.in_exp = 0; }
            for (int l = lin - depth; l < lin; ++l) o.rhs.out[l] = h->glev[l];
            o.grid = dim3((unsigned)((1ULL << lin) >> o.rhs.chunk_log));
            o.block = dim3(kRhsThreads);
            o.smem = (size_t)(1 << o.rhs.chunk_log) * 3 / 2 * sizeof(double);
            h->ops.push_back(o);
            lin -= depth;
        }
    }
    // FMG up to level Mc in the tail block
    if (Mc == M) {
        h->ops.push_back(tail_op(h, 0, nullptr, nullptr, -2 * M, nullptr, true, true));
        return;
    }
    h->ops.push_back(tail_op(h, 0, nullptr, h->glev[Mc], 0, Unext(Mc), false, false));
    cur[Mc] ^= 1;

    // one V-cycle below a level that was just restricted to Mc
    // (src: the top level's iterate when it is not in the level's own buffers)
    auto vcycle_below = [&](int top_stored, const double *src) {
        for (int l = top_stored; l > Mc;) {
            const double *u_src = (l == top_stored && src) ? src : U(l);
            int k = chainable(h, l) ? std::min(h->p.chain_down, l - Mc) : 1;
            while (k >= 2 && chain_op(h, OP_DOWN_CHAIN, l, k).block.x > (unsigned)kSweepBlockMax) --k;
            if (k >= 2) {
                // down passes of levels l .. l-k+1 in one launch; the buffers as the
                // separate passes would leave them
                Op o = chain_op(h, OP_DOWN_CHAIN, l, k);
                o.fchain.u_src = (const fx::i64 *)u_src;
                o.fchain.g[0] = (const fx::i64 *)h->glev[l];
                for (int i = 0; i < k; ++i) {
                    if (i > 0) cur[l - i] ^= 1;        // (the restriction the separate pass would store)
                    o.fchain.u_out[i] = (fx::i64 *)Unext(l - i);
                    cur[l - i] ^= 1;
                    o.fchain.g_out[i] = (fx::i64 *)h->glev[l - i - 1];
                }
                o.fchain.uc_out = (fx::i64 *)Unext(l - k);
                cur[l - k] ^= 1;
                h->ops.push_back(o);
                l -= k;
                continue;
            }
            h->ops.push_back(level_op(h, OP_DOWN, l, u_src, nullptr, Unext(l), Unext(l - 1), h->glev[l - 1]));
            cur[l] ^= 1;
            cur[l - 1] ^= 1;
            --l;
        }
        h->ops.push_back(tail_op(h, 1, (top_stored == Mc && src) ? src : U(Mc), h->glev[Mc], 0, Unext(Mc), false,
                                 false));
        cur[Mc] ^= 1;
        for (int l = Mc + 1; l <= top_stored;) {
            int k = 0;
            while (k < h->p.chain_up && l + k <= top_stored && chainable(h, l + k)) ++k;
            while (k >= 2 && chain_op(h, OP_UP_CHAIN, l, k).block.x > (unsigned)kSweepBlockMax) --k;
            if (k >= 2) {
                // up passes of levels l .. l+k-1 in one launch
                Op o = chain_op(h, OP_UP_CHAIN, l, k);
                o.fchain.uc_src = (const fx::i64 *)U(l - 1);
                for (int i = 0; i < k; ++i) {
                    o.fchain.u_in[i] = (const fx::i64 *)U(l + i);
                    o.fchain.g[i] = (const fx::i64 *)h->glev[l + i];
                    o.fchain.u_out[i] = (fx::i64 *)Unext(l + i);
                    cur[l + i] ^= 1;
                }
                h->ops.push_back(o);
                l += k;
                continue;
            }
            h->ops.push_back(level_op(h, OP_UP, l, U(l), U(l - 1), Unext(l), nullptr, nullptr));
            cur[l] ^= 1;
            ++l;
        }
    };

    const int R = M - h->nRS;          // the highest stored level below the SR levels
    // FMG steps whose top level is a stored level below the finest
    for (int k = Mc; k < (h->nRS ? R : M - 1); ++k) {
        int top = k + 1;
        h->ops.push_back(level_op(h, OP_DOWN_PI, top, U(k), nullptr, Unext(top), Unext(k), h->glev[k]));
        cur[top] ^= 1;
        cur[k] ^= 1;
        vcycle_below(k, nullptr);
        h->ops.push_back(level_op(h, OP_UP, top, U(top), U(k), Unext(top), nullptr, nullptr));
        cur[top] ^= 1;
    }
    if (h->nRS >= 1) {
        // FMG steps whose top T is an SR level (Fig. 3): the top's pre-leg from
        // Pi u_{T-1}; the SR levels below it from their assembled iterates; the
        // stored V-cycle; the post-legs (full update + compatible relaxation)
        // of the SR levels from the bottom up, the finest writing the caller's u
        // from_u: a further V-cycle on level M from the caller's current u
        // (FAS recompute: the pre-leg writes the restricted solution to uhat, keeps
        // the interpolated iterate in uold and its edge cells; the V-cycle starts
        // from uhat and the post-leg recomputes the pre-smoothed segments)
        auto sr_step = [&](int T, bool from_u) {
            const bool rcm = (h->p.post_leg == SRFMG_POST_FAS_RECOMPUTE);
            const double *gT = (T == M) ? nullptr : h->glev[T];
            double *uhat_out = rcm ? h->uhat : Unext(T - 1);
            Op pre = seg_op(h, OP_SR_PRE, T, from_u ? nullptr : U(T - 1), uhat_out, h->glev[T - 1], gT, nullptr,
                            nullptr);
            if (from_u) pre.seg_uin = TAG_U;
            if (rcm) {
                pre.seg.u_old_out = h->uold;
                pre.seg.edge_out = h->edge;
            }
            h->ops.push_back(pre);
            if (!rcm) cur[T - 1] ^= 1;
            if (h->p.tau_edge == SRFMG_TAU_ASSEMBLED)
                h->ops.push_back(seg_op(h, OP_SEAM, T, nullptr, rcm ? h->uhat : U(T - 1), h->glev[T - 1], gT, nullptr,
                                        nullptr));
            for (int L = T - 1; L > R; --L) {
                h->ops.push_back(seg_op(h, OP_SR_PRE, L, nullptr, Unext(L - 1), h->glev[L - 1], h->glev[L], U(L),
                                        nullptr));
                cur[L - 1] ^= 1;
                if (h->p.tau_edge == SRFMG_TAU_ASSEMBLED)
                    h->ops.push_back(seg_op(h, OP_SEAM, L, nullptr, U(L - 1), h->glev[L - 1], h->glev[L], nullptr,
                                            nullptr));
            }
            vcycle_below(R, rcm ? h->uhat : nullptr);
            for (int L = R + 1; L < T; ++L) {
                h->ops.push_back(seg_op(h, OP_SR_POST, L, U(L - 1), nullptr, nullptr, h->glev[L], nullptr, Unext(L)));
                cur[L] ^= 1;
            }
            if (T == M && rcm) {
                Op post = seg_op(h, OP_SR_POST, M, h->uold, nullptr, nullptr, nullptr, nullptr, nullptr);
                post.seg.uc_corr = U(M - 1);
                post.seg.uhat = h->uhat;
                post.seg.edge_in = h->edge;
                post.seg.nu_pre = h->p.nu1;
                h->ops.push_back(post);
            } else if (T == M) {
                h->ops.push_back(seg_op(h, OP_SR_POST, M, U(M - 1), nullptr, nullptr, nullptr, nullptr, nullptr));
            } else {
                h->ops.push_back(seg_op(h, OP_SR_POST, T, U(T - 1), nullptr, nullptr, h->glev[T], nullptr, Unext(T)));
                cur[T] ^= 1;
            }
        };
        for (int T = R + 1; T <= M; ++T) sr_step(T, false);
        for (int c = 0; c < h->p.n_vcycles; ++c) sr_step(M, true);
    } else {
        // level M stored in ulev[M][0]; the up pass writes the user's u
        h->ops.push_back(level_op(h, OP_DOWN_PI, M, U(M - 1), nullptr, h->ulev[M][0], Unext(M - 1),
                                  h->glev[M - 1]));
        cur[M - 1] ^= 1;
        vcycle_below(M - 1, nullptr);
        Op o = level_op(h, OP_UP, M, h->ulev[M][0], U(M - 1), nullptr, nullptr, nullptr);
        o.lev_out = TAG_U;
        h->ops.push_back(o);
        // further V-cycles (Fig. 1) from the caller's current u
        for (int c = 0; c < h->p.n_vcycles; ++c) {
            Op d = level_op(h, OP_DOWN, M, nullptr, nullptr, h->ulev[M][0], Unext(M - 1), h->glev[M - 1]);
            d.lev_uin = TAG_U;
            h->ops.push_back(d);
            cur[M - 1] ^= 1;
            vcycle_below(M - 1, nullptr);
            Op up = level_op(h, OP_UP, M, h->ulev[M][0], U(M - 1), nullptr, nullptr, nullptr);
            up.lev_out = TAG_U;
            h->ops.push_back(up);
        }
    }
}

void build_schedule(srfmg_plan *h) {
    build_schedule_ops(h);
    for (Op &o : h->ops) {
        const bool mx = (h->p.precision == SRFMG_MIXED);
        o.opk = (h->p.op == SRFMG_OP_BRATU)     ? (mx ? kOpBratuMx : kOpBratu)
                : (h->p.op == SRFMG_OP_VARCOEF) ? kOpVarcoef
                                                : kOpLaplace;
        // the variable-coefficient kernels stage their face coefficients (FP64), or
        // A, the multipliers and a second carry array (fixed point)
        const bool seg = (o.kind == OP_SR_PRE || o.kind == OP_SR_POST);
        if (op_vc(o.opk) && (o.kind == OP_DOWN || o.kind == OP_DOWN_PI || o.kind == OP_UP || seg)) {
            const size_t ml = (size_t)(seg ? o.seg.maxlen : o.lev.maxlen), mch = (size_t)(seg ? o.seg.maxch : o.lev.maxch);
            if (h->fixed) o.smem += (3 * ml + 1 + mch) * sizeof(double);
            else o.smem += ml * sizeof(double) + 2 * sizeof(double);
        }
        o.grid.y = (unsigned)h->batch;           // one grid row per problem of the batch
        if (o.kind == OP_SR_POST && o.seg.uc_corr && !h->fixed) {   // FP64 recompute: a second coarse array
            o.seg.c2_off = (int)(o.smem / sizeof(double));
            o.smem += (size_t)o.seg.maxc * sizeof(double);
        }
    }
    if (!h->fixed) return;
    for (Op &o : h->ops) to_fixed(h, o);
    Op sc = make_op(OP_SCALE);
    sc.fixed = true;
    sc.vc = (h->p.op == SRFMG_OP_VARCOEF);
    sc.scale = h->scale;
    sc.status = h->status;
    sc.level = h->M;
    // max|f| of each problem: one block per 4096 cells (at most 8 x 152)
    const size_t sblocks = std::min<size_t>(1216, std::max<size_t>(1, h->n / 4096));
    sc.grid = dim3((unsigned)sblocks, (unsigned)h->batch);
    sc.block = dim3(256);
    h->ops.insert(h->ops.begin(), sc);
}

// One kernel launch; with pdl the launch carries the programmatic-dependent-
// launch attribute (the kernel may begin launching while the preceding
// kernel of the stream runs; it waits for it in pdl_enter before touching
// data).
template <typename... KArgs, typename... Args>
cudaError_t run(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// The fixed-point kernels of one op (VC: the variable-coefficient instantiation).
template <bool VC>
cudaError_t launch_fixed_ops(const Op &o, cudaStream_t s, bool pdl) {
    cudaError_t e = cudaSuccess;
    switch (o.kind) {
    case OP_TAIL: e = run(fx::tail_kernel<VC>, o.grid, o.block, o.smem, s, pdl, o.ftail); break;
    case OP_DOWN_PI: e = run(fx::level_down_kernel<true, VC>, o.grid, o.block, o.smem, s, pdl, o.flev); break;
    case OP_DOWN: e = run(fx::level_down_kernel<false, VC>, o.grid, o.block, o.smem, s, pdl, o.flev); break;
    case OP_UP: e = run(fx::level_up_kernel<VC>, o.grid, o.block, o.smem, s, pdl, o.flev); break;
    case OP_DOWN_CHAIN: e = run(fx::level_down_chain_kernel, o.grid, o.block, o.smem, s, pdl, o.fchain); break;
    case OP_UP_CHAIN: e = run(fx::level_up_chain_kernel, o.grid, o.block, o.smem, s, pdl, o.fchain); break;
    case OP_SR_PRE: e = run(fx::sr_pre_kernel<VC>, o.grid, o.block, o.smem, s, pdl, o.fseg); break;
    case OP_SEAM: e = run(fx::seam_tau_kernel<VC>, o.grid, o.block, 0, s, pdl, o.fseg, o.nseg); break;
    case OP_SR_POST: e = run(fx::sr_post_kernel<VC>, o.grid, o.block, o.smem, s, pdl, o.fseg); break;
    default: break;
    }
    return e;
}

cudaError_t launch_fixed(const Op &o0, const Io &io, cudaStream_t s, bool pdl) {
    Op o = o0;
    const double *f = io.f;
    double *u = io.u;
    if (o.rhs_in == TAG_F) o.frhs.f = f;
    if (o.lev_g == TAG_F) o.flev.f = f;
    if (o.lev_out == TAG_U) { o.flev.u_out_f64 = u; o.flev.u_out = nullptr; }
    if (o.tail_g == TAG_F) o.ftail.f = f;
    if (o.tail_out == TAG_U) { o.ftail.u_out_f64 = u; o.ftail.u_out = nullptr; }
    if (o.seg_f == TAG_F) o.fseg.f = f;
    if (o.seg_u == TAG_U) {
        o.fseg.u_out = u;
        o.fseg.u_ref = io.u_ref;
        o.fseg.fpart = io.fout ? io.fpart : nullptr;
    }
    if (o.seg_uin == TAG_U) o.fseg.u_in_f64 = u;
    if (o.lev_uin == TAG_U) { o.flev.u_src_f64 = u; o.flev.u_src = nullptr; }
    cudaError_t e = cudaSuccess;
    switch (o.kind) {
    case OP_SCALE: {
        const long long n = (long long)o.level < 63 ? (1LL << o.level) : 0;
        e = run(fx::scale_kernel, o.grid, o.block, 0, s, pdl, f, n, o.scale, o.status, o.vc ? 1 : 0);
        break;
    }
    case OP_RHS: e = run(fx::rhs_hierarchy_kernel, o.grid, o.block, o.smem, s, pdl, o.frhs); break;
    default: e = o.vc ? launch_fixed_ops<true>(o, s, pdl) : launch_fixed_ops<false>(o, s, pdl); break;
    }
    return e;
}

// FP64 kernels of one op (NL: the Bratu instantiation).
template <int NL>
cudaError_t launch_fp64(const Op &o, cudaStream_t s, bool pdl) {
    cudaError_t e = cudaSuccess;
    switch (o.kind) {
    case OP_RHS: e = run(rhs_hierarchy_kernel, o.grid, o.block, o.smem, s, pdl, o.rhs); break;
    case OP_TAIL: e = run(tail_kernel<NL>, o.grid, o.block, o.smem, s, pdl, o.tail); break;
    case OP_DOWN_PI: e = run(level_down_kernel<true, NL>, o.grid, o.block, o.smem, s, pdl, o.lev); break;
    case OP_DOWN: e = run(level_down_kernel<false, NL>, o.grid, o.block, o.smem, s, pdl, o.lev); break;
    case OP_UP: e = run(level_up_kernel<NL>, o.grid, o.block, o.smem, s, pdl, o.lev); break;
    case OP_SR_PRE: e = run(sr_pre_kernel<NL>, o.grid, o.block, o.smem, s, pdl, o.seg); break;
    case OP_SEAM: e = run(seam_tau_kernel<NL>, o.grid, o.block, 0, s, pdl, o.seg, o.nseg); break;
    case OP_SR_POST: e = run(sr_post_kernel<NL>, o.grid, o.block, o.smem, s, pdl, o.seg); break;
    case OP_SCALE: case OP_DOWN_CHAIN: case OP_UP_CHAIN: break;
    }
    return e;
}

// Enqueue one op on s; pdl as in run().
cudaError_t launch(const Op &o0, const Io &io, cudaStream_t s, bool pdl) {
    if (o0.fixed) return launch_fixed(o0, io, s, pdl);
    Op o = o0;
    const double *f = io.f;
    double *u = io.u;
    if (o.rhs_in == TAG_F) o.rhs.in = f;
    if (o.lev_g == TAG_F) o.lev.g = f;
    if (o.lev_out == TAG_U) o.lev.u_out = u;
    if (o.tail_g == TAG_F) o.tail.g_in = f;
    if (o.tail_out == TAG_U) o.tail.u_out = u;
    if (o.seg_f == TAG_F) o.seg.f = f;
    if (o.seg_u == TAG_U) {
        o.seg.u_out = u;
        o.seg.u_ref = io.u_ref;
        o.seg.fpart = io.fout ? io.fpart : nullptr;
    }
    if (o.seg_uin == TAG_U) o.seg.u_in = u;
    if (o.lev_uin == TAG_U) o.lev.u_src = u;
    if (o.opk == kOpBratu) return launch_fp64<kOpBratu>(o, s, pdl);
    if (o.opk == kOpBratuMx) return launch_fp64<kOpBratuMx>(o, s, pdl);
    if (o.opk == kOpVarcoef) return launch_fp64<kOpVarcoef>(o, s, pdl);
    return launch_fp64<kOpLaplace>(o, s, pdl);
}

const char *kind_name(OpKind k) {
    switch (k) {
    case OP_RHS: return "rhs_hierarchy";
    case OP_TAIL: return "coarse_tail";
    case OP_DOWN_PI: return "level_down_fmg";
    case OP_DOWN: return "level_down";
    case OP_UP: return "level_up";
    case OP_SR_PRE: return "sr_pre";
    case OP_SEAM: return "seam_tau";
    case OP_SR_POST: return "sr_post";
    case OP_SCALE: return "fixed_scale";
    case OP_DOWN_CHAIN: return "level_down_chain";
    case OP_UP_CHAIN: return "level_up_chain";
    }
    return "?";
}

// Face coefficients of every level from log a (NULL: a = 1), on stream s.
cudaError_t launch_coef(srfmg_plan *h, const double *log_a, cudaStream_t s) {
    CoefArgs a;
    std::memset(&a, 0, sizeof(a));
    a.log_a = log_a;
    a.M = h->M;
    a.M0 = h->M0;
    a.bad = h->coef_bad;
    for (int l = 0; l < 32; ++l) a.out[l] = h->coef[l];
    const size_t nf = ((size_t)1 << h->M) + 1;
    const unsigned blocks = (unsigned)std::min<size_t>(4 * 152, (nf + 255) / 256);
    coef_hierarchy_kernel<<<dim3(blocks, (unsigned)h->batch), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !h->fixed) return e;
    // fixed point: the coefficient's scales per problem, then A and the multipliers of every level
    fx::CoefFxArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    for (int l = 0; l < 32; ++l) {
        fa.coef[l] = h->coef[l];
        fa.A[l] = h->fA[l];
        fa.BM[l] = h->fBM[l];
    }
    fa.sc = h->scale;
    fa.bad = h->coef_bad;
    fa.M = h->M;
    fa.M0 = h->M0;
    fx::coef_scale_kernel<<<dim3((unsigned)h->batch), 1024, 0, s>>>(fa);
    fx::coef_fixed_kernel<<<dim3(blocks, (unsigned)h->batch), 256, 0, s>>>(fa);
    return cudaGetLastError();
}

// All launches of one solve; every launch after the first overlaps its set-up
// with the preceding kernel (programmatic dependent launch).
cudaError_t enqueue_all(srfmg_plan *h, const Io &io, cudaStream_t s) {
    bool first = true;
    for (size_t i = 0; i < h->ops.size(); ++i) {
        nvtxRangePushA(h->names[i].c_str());       // one range per launch (level and kernel)
        cudaError_t e = launch(h->ops[i], io, s, !first);
        nvtxRangePop();
        if (e != cudaSuccess) return e;
        first = false;
    }
    if (io.fout)    // the segments' partials -> the functionals of each problem
        return run(functionals_finish_kernel, dim3(1, (unsigned)h->batch), dim3(kFinishThreads), 0, s, true,
                   (const double *)io.fpart, (int)(h->n / h->W), h->M, io.fout, h->status);
    return cudaSuccess;
}

// Every kernel may use up to the device's opt-in shared-memory limit; the
// attribute is per function and shared by all plans, so it is set to the
// maximum rather than to one plan's need.
srfmg_status set_smem_limits(srfmg_plan *h) {
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceGetAttribute");
    size_t need = 0;
    for (const Op &o : h->ops) need = std::max(need, o.smem);
    if (need > (size_t)optin) return fail(h, SRFMG_EUNSUPPORTED, "shared memory need exceeds the device limit");
#define SRFMG_FP64_KERNELS(OPK)                                                                            \
    (const void *)level_down_kernel<true, OPK>, (const void *)level_down_kernel<false, OPK>,                   \
        (const void *)level_up_kernel<OPK>, (const void *)sr_pre_kernel<OPK>, (const void *)sr_post_kernel<OPK>, \
        (const void *)tail_kernel<OPK>
    const void *fns[] = {SRFMG_FP64_KERNELS(kOpLaplace), SRFMG_FP64_KERNELS(kOpVarcoef), SRFMG_FP64_KERNELS(kOpBratu),
                         SRFMG_FP64_KERNELS(kOpBratuMx),
                         (const void *)rhs_hierarchy_kernel,
                         (const void *)fx::level_down_kernel<true, false>, (const void *)fx::level_down_kernel<false, false>,
                         (const void *)fx::level_up_kernel<false>, (const void *)fx::sr_pre_kernel<false>,
                         (const void *)fx::sr_post_kernel<false>, (const void *)fx::tail_kernel<false>,
                         (const void *)fx::level_down_kernel<true, true>, (const void *)fx::level_down_kernel<false, true>,
                         (const void *)fx::level_up_kernel<true>, (const void *)fx::sr_pre_kernel<true>,
                         (const void *)fx::sr_post_kernel<true>, (const void *)fx::tail_kernel<true>,
                         (const void *)fx::rhs_hierarchy_kernel, (const void *)fx::level_down_chain_kernel,
                         (const void *)fx::level_up_chain_kernel};
    for (const void *fn : fns) {
        // the opt-in limit covers static and dynamic shared memory together
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncGetAttributes");
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
    }
    return SRFMG_OK;
}

void release(srfmg_plan *h) {
    for (auto &g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t ev : {h->ev_join, h->ev_in[0], h->ev_in[1], h->ev_solved[0], h->ev_solved[1],
                           h->ev_out[0], h->ev_out[1]})
        if (ev) cudaEventDestroy(ev);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (void *ptr : h->allocs) cudaFree(ptr);
    h->allocs.clear();
}

}  // namespace

extern "C" {

srfmg_status srfmg_default_params(int32_t log2_n, srfmg_params *p) {
    if (!p) return fail(nullptr, SRFMG_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->op = SRFMG_OP_LAPLACE;
    p->precision = SRFMG_FP64;
    p->log2_n = log2_n;
    p->log2_n_coarsest = 2;
    p->n_sr_levels = 1;
    long long N = (log2_n >= 0 && log2_n < 62) ? (1LL << log2_n) : 0;
    long long W = N / 4 < 4096 ? N / 4 : 4096;
    p->segment_width = (int32_t)(W < 16 ? 16 : W);
    p->buffer_width = 8;
    p->nu1 = 1;
    p->nu2 = 1;
    p->smoother = SRFMG_SMOOTH_LEX;
    return SRFMG_OK;
}

srfmg_status srfmg_create(const srfmg_params *p, int device, srfmg_handle *out) {
    if (!out) return fail(nullptr, SRFMG_EINVAL, "out is NULL");
    *out = nullptr;
    std::string msg = check_params(p);
    if (!msg.empty()) return fail(nullptr, SRFMG_EINVAL, msg);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, SRFMG_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    if (device < 0 || device >= ndev) return fail(nullptr, SRFMG_EINVAL, "device index out of range");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, SRFMG_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));

    srfmg_plan *h = new srfmg_plan();
    h->p = *p;
    h->device = device;
    h->M = p->log2_n;
    h->M0 = p->log2_n_coarsest;
    h->nRS = p->n_sr_levels;
    h->W = p->segment_width;
    h->b = p->buffer_width;
    h->n = (size_t)1 << h->M;
    h->batch = p->batch > 0 ? p->batch : 1;
    int top_stored = h->M - h->nRS;
    const int tail_max = p->tail_level ? p->tail_level : kMaxTailLevel;
    h->Mc = top_stored < tail_max ? top_stored : tail_max;
    // further V-cycles without SR start from the caller's u with a down pass of
    // the finest level, which must then be a stored level
    if (h->nRS == 0 && p->n_vcycles > 0 && h->Mc >= h->M) h->Mc = h->M - 1;
    if (h->Mc < h->M0) h->Mc = h->M0;
    // the 64-bit fixed-point kernels serve the constant-coefficient operator; the
    // mixed precision of the other two is their FP64 kernels with FP32 corrections
    h->fixed = (p->precision == SRFMG_MIXED && p->op != SRFMG_OP_BRATU);
    const char *env = std::getenv("SRFMG_NO_GRAPH");
    h->use_graph = !(env && env[0] == '1');

    srfmg_status st = SRFMG_OK;
    const size_t B = (size_t)h->batch;   // every per-problem array holds B problems back to back
    for (int l = h->Mc; l <= h->M && st == SRFMG_OK; ++l) {
        if (l == h->M) {
            if (h->nRS == 0 && h->Mc < h->M) st = alloc_dev(h, &h->ulev[l][0], B << l);
            break;
        }
        st = alloc_dev(h, &h->ulev[l][0], B << l);
        if (st == SRFMG_OK) st = alloc_dev(h, &h->ulev[l][1], B << l);
        if (st == SRFMG_OK) st = alloc_dev(h, &h->glev[l], B << l);
    }
    if (st == SRFMG_OK && h->nRS >= 1) st = alloc_dev(h, &h->seam, B * (h->n / h->W) * 6);
    if (st == SRFMG_OK && p->post_leg == SRFMG_POST_FAS_RECOMPUTE) {
        st = alloc_dev(h, &h->uold, B * (h->n / 2));
        if (st == SRFMG_OK) st = alloc_dev(h, &h->uhat, B * (h->n / 2));
        if (st == SRFMG_OK) st = alloc_dev(h, &h->edge, B * (h->n / h->W) * 2 * (size_t)(h->b + 1));
    }
    if (st == SRFMG_OK && h->nRS >= 1) st = alloc_dev(h, &h->fpart, B * (h->n / h->W) * kNumFunc);
    if (st == SRFMG_OK && h->fixed) {
        double *sc = nullptr;
        static_assert(sizeof(fx::Scale) % sizeof(double) == 0, "Scale is a whole number of doubles");
        st = alloc_dev(h, &sc, B * (sizeof(fx::Scale) / sizeof(double)));
        h->scale = (fx::Scale *)sc;
        // the scale kernel's accumulators start at zero (it restores them after every solve)
        if (st == SRFMG_OK && (e = cudaMemset(sc, 0, B * sizeof(fx::Scale))) != cudaSuccess)
            st = cuda_fail(h, e, "cudaMemset(scales)");
    }
    if (p->op == SRFMG_OP_VARCOEF) {
        for (int l = h->M0; l <= h->M && st == SRFMG_OK; ++l) st = alloc_dev(h, &h->coef[l], B * (((size_t)1 << l) + 1));
        for (int l = h->M0; l <= h->M && st == SRFMG_OK && h->fixed; ++l) {
            double *w = nullptr;
            st = alloc_dev(h, &w, B * (((size_t)1 << l) + 1));
            h->fA[l] = (fx::u64 *)w;
            if (st == SRFMG_OK) st = alloc_dev(h, &w, B * ((size_t)2 << l));
            h->fBM[l] = (fx::u64 *)w;
        }
        double *flag = nullptr;
        if (st == SRFMG_OK) st = alloc_dev(h, &flag, 1);
        h->coef_bad = (int *)flag;
    }
    if (st == SRFMG_OK) {
        double *w = nullptr;
        st = alloc_dev(h, &w, 1);
        h->status = (int *)w;
        if (st == SRFMG_OK && (e = cudaMemset(w, 0, sizeof(double))) != cudaSuccess) st = cuda_fail(h, e, "cudaMemset");
    }
    if (st == SRFMG_OK && p->op == SRFMG_OP_BRATU && p->precision == SRFMG_MIXED &&
        (e = upload_exp_table()) != cudaSuccess)
        st = cuda_fail(h, e, "exponential table");
    const int n0 = 1 << h->M0;
    if (st == SRFMG_OK) st = alloc_dev(h, &h->Ainv, (size_t)n0 * n0);
    if (st == SRFMG_OK) {
        std::vector<double> inv = coarsest_inverse(n0);
        e = cudaMemcpy(h->Ainv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMemcpy(coarsest inverse)");
    }
    if (st == SRFMG_OK) {
        build_schedule(h);
        for (const Op &o : h->ops)
            h->names.push_back(std::string(o.fixed ? "fx." : "") + kind_name(o.kind) + " L" + std::to_string(o.level));
        st = set_smem_limits(h);
    }
    if (st == SRFMG_OK) {
        e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaStreamCreate");
    }
    if (st == SRFMG_OK && p->op == SRFMG_OP_VARCOEF) {          // a = 1 until srfmg_set_coefficient
        // (after the workspace memsets on the legacy stream, which the capture
        // stream does not wait for: the fixed-point scales are written here)
        e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = launch_coef(h, nullptr, h->cap_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->cap_stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "coefficient initialisation");
    }
    if (st != SRFMG_OK) {
        g_create_error = h->err;
        release(h);
        delete h;
        return st;
    }
    *out = h;
    return SRFMG_OK;
}

}  // extern "C"

namespace {

// Enqueue one solve with the caller's pointers io (checked by the caller):
// replay the captured graph of this pointer set, capturing it first.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

srfmg_status solve_io(srfmg_handle h, const Io &io, cudaStream_t s) {
    NvtxRange range(io.fout ? "srfmg_solve_functionals" : "srfmg_solve");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (!h->use_graph) {
        e = enqueue_all(h, io, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
        h->solved = true;
        return SRFMG_OK;
    }
    srfmg_plan::GraphSlot *slot = nullptr;
    for (auto &g : h->graphs)
        if (g.exec && g.f == io.f && g.u == io.u && g.u_ref == io.u_ref && g.fout == io.fout) slot = &g;
    if (!slot) {
        slot = &h->graphs[0];
        for (auto &g : h->graphs)
            if (!g.exec || g.used < slot->used) slot = &g;
        if (slot->exec) { cudaGraphExecDestroy(slot->exec); slot->exec = nullptr; }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
        cudaError_t le = enqueue_all(h, io, h->cap_stream);
        e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (le != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(h, le, "kernel launch during capture"); }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&slot->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { slot->exec = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
        slot->f = io.f;
        slot->u = io.u;
        slot->u_ref = io.u_ref;
        slot->fout = io.fout;
    }
    slot->used = ++h->graph_clock;
    e = cudaGraphLaunch(slot->exec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    h->solved = true;
    return SRFMG_OK;
}

// [p, p + n) and [q, q + m) share memory
bool overlap(const void *p, size_t pn, const void *q, size_t qn) {
    const char *a = (const char *)p, *b = (const char *)q;
    return a < b + qn && b < a + pn;
}

}  // namespace

extern "C" {

srfmg_status srfmg_solve(srfmg_handle h, const double *f, double *u, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (!f || !u) return fail(h, SRFMG_EINVAL, "f and u must be device pointers");
    if (((uintptr_t)f & 15) || ((uintptr_t)u & 15)) return fail(h, SRFMG_EINVAL, "f and u must be 16-byte aligned");
    const size_t bytes = h->n * (size_t)h->batch * sizeof(double);
    if (overlap(f, bytes, u, bytes)) return fail(h, SRFMG_EINVAL, "f and u overlap");
    return solve_io(h, Io{f, u, nullptr, nullptr, nullptr}, (cudaStream_t)stream);
}

srfmg_status srfmg_solve_functionals(srfmg_handle h, const double *f, double *u, const double *u_ref,
                                     double *functionals, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (h->nRS < 1)
        return fail(h, SRFMG_EUNSUPPORTED, "functionals are collected by the SR post-leg: the plan needs an SR level");
    if (!f || !functionals) return fail(h, SRFMG_EINVAL, "f and functionals must be device pointers");
    if (!u && h->p.n_vcycles > 0)
        return fail(h, SRFMG_EINVAL, "a plan with n_vcycles > 0 needs u: each V-cycle starts from the fine solution");
    if (((uintptr_t)f & 15) || ((uintptr_t)u & 15) || ((uintptr_t)u_ref & 7) || ((uintptr_t)functionals & 7))
        return fail(h, SRFMG_EINVAL, "f and u must be 16-byte aligned, u_ref and functionals 8-byte aligned");
    const size_t bytes = h->n * (size_t)h->batch * sizeof(double);
    const size_t fbytes = (size_t)kNumFunc * h->batch * sizeof(double);
    if ((u && overlap(f, bytes, u, bytes)) || (u && u_ref && overlap(u, bytes, u_ref, bytes)) ||
        overlap(functionals, fbytes, f, bytes) || (u && overlap(functionals, fbytes, u, bytes)) ||
        (u_ref && overlap(functionals, fbytes, u_ref, bytes)))
        return fail(h, SRFMG_EINVAL, "an output overlaps another argument");
    return solve_io(h, Io{f, u, u_ref, functionals, h->fpart}, (cudaStream_t)stream);
}

srfmg_status srfmg_reconstruct(srfmg_handle h, const double *f, int32_t seg_begin, int32_t seg_count,
                               double *u_seg, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (h->nRS < 1) return fail(h, SRFMG_EUNSUPPORTED, "reconstruction expands SR segments: the plan needs an SR level");
    if (h->p.post_leg == SRFMG_POST_FAS_RECOMPUTE)
        return fail(h, SRFMG_EUNSUPPORTED, "reconstruction rebuilds segments by the full update (SRFMG_POST_FULL_UPDATE)");
    if (!h->solved) return fail(h, SRFMG_EINVAL, "no solve has been enqueued on this plan");
    const int nseg = (int)(h->n / h->W);
    if (seg_begin < 0 || seg_count < 1 || seg_begin > nseg - seg_count)
        return fail(h, SRFMG_EINVAL, "segments [seg_begin, seg_begin + seg_count) must lie in [0, n_segments)");
    if (!f || !u_seg) return fail(h, SRFMG_EINVAL, "f and u_seg must be device pointers");
    if (((uintptr_t)f & 15) || ((uintptr_t)u_seg & 7))
        return fail(h, SRFMG_EINVAL, "f must be 16-byte aligned, u_seg 8-byte aligned");
    const size_t fb = h->n * (size_t)h->batch * sizeof(double);
    const size_t ub = (size_t)seg_count * h->W * h->batch * sizeof(double);
    if (overlap(f, fb, u_seg, ub)) return fail(h, SRFMG_EINVAL, "f and u_seg overlap");
    const Op *post = nullptr;
    for (const Op &o : h->ops)
        if (o.kind == OP_SR_POST) post = &o;
    if (!post) return fail(h, SRFMG_EUNSUPPORTED, "the plan has no SR post-leg");
    Op o = *post;
    o.grid.x = (unsigned)seg_count;
    o.seg.seg0 = seg_begin;
    o.fseg.seg0 = seg_begin;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = launch(o, Io{f, u_seg, nullptr, nullptr, nullptr}, (cudaStream_t)stream, false);
    return e == cudaSuccess ? SRFMG_OK : cuda_fail(h, e, "reconstruction kernel");
}

srfmg_status srfmg_solve_host(srfmg_handle h, const double *f, double *u, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (!f || !u) return fail(h, SRFMG_EINVAL, "f and u must be host pointers");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t total = h->n * (size_t)h->batch;
    if (!h->f_stage) {
        srfmg_status st = alloc_dev(h, &h->f_stage, total);
        if (st == SRFMG_OK) st = alloc_dev(h, &h->u_stage, total);
        if (st != SRFMG_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(h->f_stage, f, total * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync(f)");
    srfmg_status st = srfmg_solve(h, h->f_stage, h->u_stage, stream);
    if (st != SRFMG_OK) return st;
    e = cudaMemcpyAsync(u, h->u_stage, total * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync(u)");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return SRFMG_OK;
}

srfmg_status srfmg_solve_host_async(srfmg_handle h, const double *f, double *u, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (!f || !u) return fail(h, SRFMG_EINVAL, "f and u must be host pointers");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t total = h->n * (size_t)h->batch, bytes = total * sizeof(double);
    if (!h->s_out) {            // first call: staging pairs, streams and events
        srfmg_status st = SRFMG_OK;
        for (int b = 0; b < 2 && st == SRFMG_OK; ++b) {
            st = alloc_dev(h, &h->hf[b], total);
            if (st == SRFMG_OK) st = alloc_dev(h, &h->hu[b], total);
        }
        if (st != SRFMG_OK) return st;
        cudaEvent_t *evs[] = {&h->ev_join, &h->ev_in[0], &h->ev_in[1], &h->ev_solved[0],
                              &h->ev_solved[1], &h->ev_out[0], &h->ev_out[1]};
        for (cudaEvent_t *ev : evs)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline set-up");
    }
    const int b = h->hslot;
    h->hslot ^= 1;
    cudaStream_t s = (cudaStream_t)stream;
    // copy in as soon as the solve that last read this staging buffer (two
    // calls back) is done; f is host memory, ready when the call is made, so
    // the copy does not wait for `stream` (it overlaps the previous solve)
    e = cudaStreamWaitEvent(h->s_in, h->ev_solved[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hf[b], f, bytes, cudaMemcpyHostToDevice, h->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[b], h->s_in);
    // solve on `stream` once f is in and this solution buffer's last copy-out is done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_in[b], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_out[b], 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline (copy in)");
    srfmg_status st = srfmg_solve(h, h->hf[b], h->hu[b], stream);
    if (st != SRFMG_OK) return st;
    // copy out after the solve, overlapping the next call's solve
    e = cudaEventRecord(h->ev_solved[b], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_solved[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, h->hu[b], bytes, cudaMemcpyDeviceToHost, h->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[b], h->s_out);
    if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline (copy out)");
    return SRFMG_OK;
}

srfmg_status srfmg_solve_host_join(srfmg_handle h, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (!h->s_out) return SRFMG_OK;        // nothing was enqueued
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, h->ev_join, 0);
    return e == cudaSuccess ? SRFMG_OK : cuda_fail(h, e, "srfmg_solve_host_join");
}

// The operator of SRFMG_OP_LAPLACE (cell-centred, odd ghosts: tridiag(-1, 2, -1)/h^2
// with 3 in the wall rows) is symmetric, so the adjoint equation L^T lambda = dL/du is
// the forward equation with dL/du as its right-hand side: lambda = dL/df comes from
// the same FMG(-SR) solve.
srfmg_status srfmg_adjoint(srfmg_handle h, const double *dL_du, double *dL_df, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    // -(a u')' is symmetric as well; the Bratu operator is nonlinear
    if (h->p.op == SRFMG_OP_BRATU) return fail(h, SRFMG_EUNSUPPORTED, "adjoint of this operator");
    return srfmg_solve(h, dL_du, dL_df, stream);
}

srfmg_status srfmg_coef_gradient(srfmg_handle h, const double *u, const double *lam, double *dL_dloga,
                                 void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (h->p.op != SRFMG_OP_VARCOEF) return fail(h, SRFMG_EINVAL, "the plan's operator has no coefficient");
    if (!u || !lam || !dL_dloga) return fail(h, SRFMG_EINVAL, "u, lam and dL_dloga must be device pointers");
    if (((uintptr_t)u | (uintptr_t)lam | (uintptr_t)dL_dloga) & 7)
        return fail(h, SRFMG_EINVAL, "u, lam and dL_dloga must be 8-byte aligned");
    const size_t cells = h->n * (size_t)h->batch, faces = (h->n + 1) * (size_t)h->batch;
    const double *o = dL_dloga;
    if ((o < u + cells && u < o + faces) || (o < lam + cells && lam < o + faces))
        return fail(h, SRFMG_EINVAL, "dL_dloga overlaps u or lam");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const unsigned blocks = (unsigned)std::min<size_t>(4 * 152, (h->n + 1 + 255) / 256);
    coef_gradient_kernel<<<dim3(blocks, (unsigned)h->batch), 256, 0, (cudaStream_t)stream>>>(
        u, lam, h->coef[h->M], dL_dloga, h->M);
    e = cudaGetLastError();
    return e == cudaSuccess ? SRFMG_OK : cuda_fail(h, e, "coefficient gradient kernel");
}

srfmg_status srfmg_set_coefficient(srfmg_handle h, const double *log_a, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    if (h->p.op != SRFMG_OP_VARCOEF) return fail(h, SRFMG_EINVAL, "the plan's operator has no coefficient");
    if (!log_a || ((uintptr_t)log_a & 7)) return fail(h, SRFMG_EINVAL, "log_a must be an 8-byte aligned device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(h->coef_bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_coef(h, log_a, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, h->coef_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "coefficient kernel");
    if (!bad) return SRFMG_OK;
    // rejected: back to a = 1, so that no solve runs on a coefficient the sweeps cannot take
    e = launch_coef(h, nullptr, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "coefficient reset");
    return fail(h, SRFMG_EINVAL,
                "log_a: a value is not finite or beyond +-700, or adjacent faces of a level of 128 or more "
                "cells differ by more than a factor 1.5 (ln 1.5 in log a), or (SRFMG_MIXED) max a / min a is "
                "2^8 or more; the coefficient was reset to a = 1");
}

srfmg_status srfmg_check(srfmg_handle h, void *stream) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int word = 0;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&word, h->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "srfmg_check");
    if (word & kStatusNonFinite)
        return fail(h, SRFMG_ENONFINITE, "a non-finite value was found in f or in the functionals since the last check");
    return SRFMG_OK;
}

srfmg_status srfmg_query(srfmg_handle h, srfmg_info *info) {
    if (!h || !info) return fail(h, SRFMG_EINVAL, "handle or info is NULL");
    std::memset(info, 0, sizeof(*info));
    info->workspace_bytes = (int64_t)h->ws_bytes;
    info->kernels_per_solve = (int32_t)h->ops.size();
    info->coarse_tail_level = h->Mc;
    info->n_segments = h->nRS ? (int32_t)(h->n / h->W) : 0;
    info->segment_width = h->nRS ? h->W : 0;
    info->buffer_width = h->nRS ? h->b : 0;
    info->batch = h->batch;
    return SRFMG_OK;
}

srfmg_status srfmg_profile(srfmg_handle h, const double *f, double *u, void *stream,
                           int32_t nsolves, float *ms_per_launch, int32_t capacity) {
    if (!h) return fail(nullptr, SRFMG_EINVAL, "handle is NULL");
    const int nops = (int)h->ops.size();
    if (!f || !u || !ms_per_launch || capacity < nops || nsolves < 1)
        return fail(h, SRFMG_EINVAL, "bad arguments to srfmg_profile");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev((size_t)nops * nsolves * 2, nullptr);
    for (auto &x : ev) {
        e = cudaEventCreate(&x);
        if (e != cudaSuccess) break;
    }
    for (int k = 0; k < nsolves && e == cudaSuccess; ++k)
        for (int i = 0; i < nops && e == cudaSuccess; ++i) {
            size_t idx = ((size_t)k * nops + i) * 2;
            e = cudaEventRecord(ev[idx], s);
            nvtxRangePushA(h->names[i].c_str());
            if (e == cudaSuccess) e = launch(h->ops[i], Io{f, u, nullptr, nullptr, nullptr}, s, false);
            nvtxRangePop();
            if (e == cudaSuccess) e = cudaEventRecord(ev[idx + 1], s);
        }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int i = 0; i < nops && e == cudaSuccess; ++i) {
        double acc = 0.0;
        for (int k = 0; k < nsolves; ++k) {
            size_t idx = ((size_t)k * nops + i) * 2;
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[idx], ev[idx + 1]);
            acc += ms;
        }
        ms_per_launch[i] = (float)(acc / nsolves);
    }
    for (auto &x : ev) if (x) cudaEventDestroy(x);
    return e == cudaSuccess ? SRFMG_OK : cuda_fail(h, e, "srfmg_profile");
}

const char *srfmg_launch_name(srfmg_handle h, int32_t i) {
    if (!h || i < 0 || i >= (int32_t)h->names.size()) return nullptr;
    return h->names[i].c_str();
}

srfmg_status srfmg_destroy(srfmg_handle h) {
    if (!h) return SRFMG_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    release(h);
    delete h;
    return SRFMG_OK;
}

const char *srfmg_last_error(srfmg_handle h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace {

// Time a plan per candidate parameter set (two warm-up solves of a zero right-
// hand side, then reps timed ones, CUDA events on a stream of its own) and
// return the fastest in *best; ms[k] receives candidate k's milliseconds per solve.
srfmg_status time_candidates(const std::vector<srfmg_params> &cand, int device, int32_t reps, srfmg_params *best,
                             float *ms, int32_t capacity) {
    const srfmg_params *base = &cand[0];
    const long long N = 1LL << base->log2_n;
    const size_t B = (size_t)(base->batch > 0 ? base->batch : 1);
    double *f = nullptr, *u = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&f, B * (size_t)N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&u, B * (size_t)N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(f, 0, B * (size_t)N * sizeof(double));   // no data-dependent control flow
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    srfmg_status st = (e == cudaSuccess) ? SRFMG_OK : fail(nullptr, SRFMG_ECUDA, std::string("autotune set-up: ") + cudaGetErrorString(e));
    float best_ms = 0.f;
    for (size_t k = 0; k < cand.size() && st == SRFMG_OK; ++k) {
        const srfmg_params p = cand[k];
        srfmg_handle h = nullptr;
        st = srfmg_create(&p, device, &h);
        for (int w = 0; w < 2 && st == SRFMG_OK; ++w) st = srfmg_solve(h, f, u, s);
        if (st == SRFMG_OK && (e = cudaEventRecord(e0, s)) != cudaSuccess) st = SRFMG_ECUDA;
        for (int r = 0; r < reps && st == SRFMG_OK; ++r) st = srfmg_solve(h, f, u, s);
        float t = 0.f;
        if (st == SRFMG_OK && ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                               (e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess))
            st = fail(nullptr, SRFMG_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
        if (st != SRFMG_OK && h) g_create_error = h->err;
        srfmg_destroy(h);
        t /= (float)reps;
        if (st == SRFMG_OK) {
            if (ms && (int32_t)k < capacity) ms[k] = t;
            if (k == 0 || t < best_ms) { best_ms = t; *best = p; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(f);
    cudaFree(u);
    return st;
}

// The shape candidates of srfmg_autotune_shape: distinct coarse tails, then tiles.
struct Shape {
    int tail, tile, cdown, cup;
};

// The CTA shapes the shape autotuner times: every distinct coarse tail in
// 9..12 with 128, 256 or 512 cells per tile; for the fixed-point -u'' = f
// also the two finest of those tails with 256 or 512 cells per tile and
// chained passes (down chains of 2, up chains of 3 or 4 levels).
std::vector<Shape> shape_candidates(const srfmg_params *base) {
    std::vector<Shape> cand;
    std::vector<int> tails;
    const int top = base->log2_n - base->n_sr_levels;
    int prev_mc = -1;
    for (int t = 9; t <= 12; ++t) {
        if (t < base->log2_n_coarsest) continue;
        const int mc = std::max(base->log2_n_coarsest, std::min(t, top));
        if (mc == prev_mc) continue;
        prev_mc = mc;
        tails.push_back(t);
        for (int tc : {128, 256, 512}) cand.push_back({t, tc, 0, 0});
    }
    if (cand.empty()) cand.push_back({12, 256, 0, 0});
    if (base->precision == SRFMG_MIXED && base->op == SRFMG_OP_LAPLACE) {
        for (size_t i = tails.size() >= 2 ? tails.size() - 2 : 0; i < tails.size(); ++i)
            for (int tc : {256, 512})
                for (int cu : {3, 4}) cand.push_back({tails[i], tc, 2, cu});
    }
    return cand;
}

}  // namespace

extern "C" {

srfmg_status srfmg_autotune(const srfmg_params *base, int device, int32_t reps, srfmg_params *best,
                            float *ms, int32_t capacity, int32_t *ncand) {
    if (!base || !best || reps < 1 || (ms && capacity < 0)) return fail(nullptr, SRFMG_EINVAL, "bad arguments to srfmg_autotune");
    std::string msg = check_params(base);
    if (!msg.empty()) return fail(nullptr, SRFMG_EINVAL, msg);
    if (base->n_sr_levels != 1) return fail(nullptr, SRFMG_EINVAL, "srfmg_autotune tunes the SR segment layout (n_sr_levels = 1)");
    const long long N = 1LL << base->log2_n;
    std::vector<srfmg_params> cand;
    for (int W = 256; W <= 4096; W *= 2)
        for (int b : {4, 8})
            if (W <= N / 2 && b <= W) {
                srfmg_params p = *base;
                p.segment_width = W;
                p.buffer_width = b;
                cand.push_back(p);
            }
    if (cand.empty()) {
        srfmg_params p = *base;
        p.segment_width = (int)std::max<long long>(16, N);
        p.buffer_width = 4;
        cand.push_back(p);
    }
    if (ncand) *ncand = (int32_t)cand.size();
    return time_candidates(cand, device, reps, best, ms, capacity);
}

srfmg_status srfmg_autotune_shape(const srfmg_params *base, int device, int32_t reps, srfmg_params *best,
                                  float *ms, int32_t capacity, int32_t *ncand) {
    if (!base || !best || reps < 1 || (ms && capacity < 0))
        return fail(nullptr, SRFMG_EINVAL, "bad arguments to srfmg_autotune_shape");
    std::string msg = check_params(base);
    if (!msg.empty()) return fail(nullptr, SRFMG_EINVAL, msg);
    std::vector<srfmg_params> cand;
    for (const auto &c : shape_candidates(base)) {
        srfmg_params p = *base;
        p.tail_level = c.tail;
        p.tile_cells = c.tile;
        p.chain_down = c.cdown;
        p.chain_up = c.cup;
        cand.push_back(p);
    }
    if (ncand) *ncand = (int32_t)cand.size();
    return time_candidates(cand, device, reps, best, ms, capacity);
}

srfmg_status srfmg_autotune_shape_candidate(const srfmg_params *base, int32_t k, srfmg_params *cand) {
    if (!base || !cand || k < 0) return fail(nullptr, SRFMG_EINVAL, "bad arguments");
    const auto list = shape_candidates(base);
    if (k >= (int32_t)list.size()) return fail(nullptr, SRFMG_EINVAL, "candidate index out of range");
    *cand = *base;
    cand->tail_level = list[k].tail;
    cand->tile_cells = list[k].tile;
    cand->chain_down = list[k].cdown;
    cand->chain_up = list[k].cup;
    return SRFMG_OK;
}

srfmg_status srfmg_autotune_candidate(const srfmg_params *base, int32_t k, int32_t *segment_width,
                                      int32_t *buffer_width) {
    if (!base || !segment_width || !buffer_width || k < 0) return fail(nullptr, SRFMG_EINVAL, "bad arguments");
    const long long N = 1LL << base->log2_n;
    int32_t i = 0;
    for (int W = 256; W <= 4096; W *= 2)
        for (int b : {4, 8})
            if (W <= N / 2 && b <= W) {
                if (i == k) { *segment_width = W; *buffer_width = b; return SRFMG_OK; }
                ++i;
            }
    if (i == 0 && k == 0) { *segment_width = (int32_t)std::max<long long>(16, N); *buffer_width = 4; return SRFMG_OK; }
    return fail(nullptr, SRFMG_EINVAL, "candidate index out of range");
}

const char *srfmg_version(void) { return "srfmg 0.1 sm_103a"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Throughput probes for the roofline denominators of the arithmetic-bound
// kernels.  Each thread runs eight interleaved dependent chains (enough
// independent work per warp to hide the pipe latency); the chains feed one
// another, so no chain can be folded into a closed form, and every thread
// writes its result.  Per chain step: one 64-bit add (i64_add), two 64-bit adds
// and a 64-bit arithmetic shift (i64_avg: (x + y + 1) >> 1, the rounding halving
// of the fixed-point sweep), one FP64 or one FP32 fused multiply-add.
// ---------------------------------------------------------------------------
namespace {

constexpr int kProbeChains = 8;

__global__ void probe_i64_add(long long *out, int iters) {
    long long a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = threadIdx.x * 7 + k + blockIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] += a[(k + 1) % kProbeChains];
    }
    long long r = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) r ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void probe_i64_avg(long long *out, int iters) {
    long long a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = ((long long)(threadIdx.x * 7 + k + blockIdx.x)) << 40;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = (a[k] + a[(k + 1) % kProbeChains] + 1) >> 1;
    }
    long long r = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) r ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void probe_dfma(double *out, int iters) {
    double a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    const double x = 0.999999, y = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], x, y);
    }
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) r += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void probe_ffma(double *out, int iters) {
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
    const float x = 0.9999f, y = 1e-5f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], x, y);
    }
    float r = 0.0f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) r += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace

extern "C" {

srfmg_status srfmg_exp_error(int device, double lo, double hi, int32_t n, double *max_rel) {
    if (!max_rel || n < 1 || n > (1 << 26) || !(lo <= hi) || !(fabs(lo) <= 700.0) || !(fabs(hi) <= 700.0))
        return fail(nullptr, SRFMG_EINVAL, "bad arguments to srfmg_exp_error");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, SRFMG_ECUDA, "no CUDA device");
    }
    if (device < 0 || device >= ndev) return fail(nullptr, SRFMG_EINVAL, "device index out of range");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    if ((e = upload_exp_table()) != cudaSuccess) return cuda_fail(nullptr, e, "exponential table");
    unsigned long long *d = nullptr;
    if ((e = cudaMalloc(&d, sizeof(*d))) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, SRFMG_ENOMEM, "cudaMalloc");
    }
    unsigned long long bits = 0;
    e = cudaMemset(d, 0, sizeof(*d));
    if (e == cudaSuccess) {
        exp_error_kernel<<<std::min(1216, (n + 255) / 256), 256>>>(lo, hi, n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "srfmg_exp_error");
    std::memcpy(max_rel, &bits, sizeof(double));
    return SRFMG_OK;
}

srfmg_status srfmg_alu_peaks(int device, double *ops_per_s) {
    if (!ops_per_s) return fail(nullptr, SRFMG_EINVAL, "ops_per_s is NULL");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, SRFMG_ECUDA, "no CUDA device");
    }
    if (device < 0 || device >= ndev) return fail(nullptr, SRFMG_EINVAL, "device index out of range");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 256, blocks = 8 * (sms > 0 ? sms : 1);
    const size_t nthr = (size_t)threads * blocks;
    void *buf = nullptr;
    if ((e = cudaMalloc(&buf, nthr * sizeof(double))) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, SRFMG_ENOMEM, "cudaMalloc(probe)");
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // (iterations, operations per chain step) of each probe
    const int iters[4] = {4096, 2048, 256, 8192};
    const double ops_per_step[4] = {1.0, 3.0, 2.0, 2.0};   // adds; adds + shift; flops of an FMA
    srfmg_status rc = SRFMG_OK;
    for (int p = 0; p < 4 && rc == SRFMG_OK; ++p) {
        float best = 1e30f;
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(e0, st);
            switch (p) {
            case 0: probe_i64_add<<<blocks, threads, 0, st>>>((long long *)buf, iters[p]); break;
            case 1: probe_i64_avg<<<blocks, threads, 0, st>>>((long long *)buf, iters[p]); break;
            case 2: probe_dfma<<<blocks, threads, 0, st>>>((double *)buf, iters[p]); break;
            default: probe_ffma<<<blocks, threads, 0, st>>>((double *)buf, iters[p]); break;
            }
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
                rc = cuda_fail(nullptr, e, "throughput probe");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;      // the first run warms up
        }
        ops_per_s[p] = (double)nthr * iters[p] * kProbeChains * ops_per_step[p] / (best * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(buf);
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Groups: independent problems of uneven sizes, one batched plan per size,
// all plans replayed as one CUDA graph with a branch per plan.
// ---------------------------------------------------------------------------
struct srfmg_group {
    int device = 0;
    std::vector<srfmg_plan *> plans;       // ascending size
    std::vector<int> m, count;             // size and problems of each plan
    std::vector<size_t> off;               // first cell of each plan's part
    size_t total = 0;
    cudaStream_t cap = nullptr;            // capture origin
    std::vector<cudaStream_t> side;        // one branch per plan
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;        // captured for (gf, gu)
    const double *gf = nullptr;
    double *gu = nullptr;
    bool use_graph = true;
    double *f_stage = nullptr, *u_stage = nullptr;
    std::string err = "no error";
};

namespace {

constexpr int kGroupPlanMax = 65535;       // problems per plan (grid rows)
thread_local std::string g_group_create_error = "no error";

srfmg_status gfail(srfmg_group *g, srfmg_status st, const std::string &msg) {
    if (g) g->err = msg; else g_group_create_error = msg;
    return st;
}

// Problem order of the packed layout: by size, then by index.
std::vector<int> group_order(int32_t nprob, const int32_t *log2_n) {
    std::vector<int> idx(nprob);
    for (int k = 0; k < nprob; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return log2_n[a] < log2_n[b]; });
    return idx;
}

void group_release(srfmg_group *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (cudaEvent_t e : g->join) if (e) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    for (cudaStream_t s : g->side) if (s) cudaStreamDestroy(s);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->f_stage) cudaFree(g->f_stage);
    if (g->u_stage) cudaFree(g->u_stage);
    for (srfmg_plan *h : g->plans) srfmg_destroy(h);
    g->plans.clear();
}

// Fork from s into one branch per plan, enqueue each plan's launches on its
// branch, join back into s.  Under capture this records the group's graph.
cudaError_t group_enqueue(srfmg_group *g, const double *f, double *u, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(g->fork, s);
    for (size_t c = 0; c < g->plans.size() && e == cudaSuccess; ++c) {
        e = cudaStreamWaitEvent(g->side[c], g->fork, 0);
        if (e == cudaSuccess)
            e = enqueue_all(g->plans[c], Io{f + g->off[c], u + g->off[c], nullptr, nullptr, nullptr}, g->side[c]);
        if (e == cudaSuccess) e = cudaEventRecord(g->join[c], g->side[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g->join[c], 0);
    }
    return e;
}

}  // namespace

extern "C" {

srfmg_status srfmg_group_offsets(int32_t nprob, const int32_t *log2_n, int64_t *offsets) {
    if (nprob < 1 || !log2_n || !offsets) return gfail(nullptr, SRFMG_EINVAL, "nprob must be >= 1 and the arrays non-NULL");
    for (int k = 0; k < nprob; ++k)
        if (log2_n[k] < 1 || log2_n[k] > 28) return gfail(nullptr, SRFMG_EINVAL, "every log2_n must be in [1, 28]");
    int64_t at = 0;
    for (int k : group_order(nprob, log2_n)) {
        offsets[k] = at;
        at += (int64_t)1 << log2_n[k];
    }
    offsets[nprob] = at;
    return SRFMG_OK;
}

srfmg_status srfmg_group_create(const srfmg_params *base, int32_t nprob, const int32_t *log2_n, int32_t tune,
                                int device, srfmg_group_handle *out) {
    if (!out) return gfail(nullptr, SRFMG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!base || tune < 0) return gfail(nullptr, SRFMG_EINVAL, "base is NULL or tune < 0");
    std::vector<int64_t> offs((size_t)std::max(nprob, 0) + 1);
    if (srfmg_group_offsets(nprob, log2_n, offs.data()) != SRFMG_OK) return SRFMG_EINVAL;
    if (tune > 0 && base->n_sr_levels != 1)
        return gfail(nullptr, SRFMG_EINVAL, "tune > 0 tunes the SR segment layout (n_sr_levels = 1)");
    // the plans: runs of equal size in the packed order, at most kGroupPlanMax problems each
    std::vector<int> order = group_order(nprob, log2_n);
    std::vector<srfmg_params> ps;
    std::vector<int> pm, pcount;
    std::vector<size_t> poff;
    for (size_t i = 0; i < order.size();) {
        const int mk = log2_n[order[i]];
        size_t j = i;
        while (j < order.size() && log2_n[order[j]] == mk && j - i < (size_t)kGroupPlanMax) ++j;
        srfmg_params p = *base;
        p.log2_n = mk;
        p.batch = (int32_t)(j - i);
        if (p.n_sr_levels >= 1) {
            const int N = 1 << mk;
            p.segment_width = std::min(base->segment_width, std::max(16, N / 4));
            p.buffer_width = std::min(base->buffer_width, p.segment_width);
        }
        std::string msg = check_params(&p);
        if (!msg.empty()) return gfail(nullptr, SRFMG_EINVAL, "size 2^" + std::to_string(mk) + ": " + msg);
        ps.push_back(p);
        pm.push_back(mk);
        pcount.push_back((int)(j - i));
        poff.push_back((size_t)offs[order[i]]);
        i = j;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return gfail(nullptr, SRFMG_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    if (device < 0 || device >= ndev) return gfail(nullptr, SRFMG_EINVAL, "device index out of range");
    srfmg_group *g = new srfmg_group();
    g->device = device;
    g->total = (size_t)offs[nprob];
    const char *env = std::getenv("SRFMG_NO_GRAPH");
    g->use_graph = !(env && env[0] == '1');
    srfmg_status st = SRFMG_OK;
    for (size_t c = 0; c < ps.size() && st == SRFMG_OK; ++c) {
        srfmg_params p = ps[c];
        if (tune > 0) {          // the layout of this size, timed on a sample of its problems
            srfmg_params probe = p, best;
            const int sample = std::max(1, (1 << 24) >> pm[c]);
            probe.batch = std::min(pcount[c], sample);
            st = srfmg_autotune(&probe, device, tune, &best, nullptr, 0, nullptr);
            if (st != SRFMG_OK) { st = gfail(g, st, "autotune of size 2^" + std::to_string(pm[c]) + ": " + g_create_error); break; }
            p.segment_width = best.segment_width;
            p.buffer_width = best.buffer_width;
            // then its CTA shape (coarse tail extent, tile cells) with that layout
            probe.segment_width = p.segment_width;
            probe.buffer_width = p.buffer_width;
            st = srfmg_autotune_shape(&probe, device, tune, &best, nullptr, 0, nullptr);
            if (st != SRFMG_OK) { st = gfail(g, st, "shape autotune of size 2^" + std::to_string(pm[c]) + ": " + g_create_error); break; }
            p.tail_level = best.tail_level;
            p.tile_cells = best.tile_cells;
            p.chain_down = best.chain_down;
            p.chain_up = best.chain_up;
        }
        srfmg_handle h = nullptr;
        st = srfmg_create(&p, device, &h);
        if (st != SRFMG_OK) { st = gfail(g, st, "plan of size 2^" + std::to_string(pm[c]) + ": " + g_create_error); break; }
        g->plans.push_back(h);
        g->m.push_back(pm[c]);
        g->count.push_back(pcount[c]);
        g->off.push_back(poff[c]);
    }
    if (st == SRFMG_OK) {
        e = cudaSetDevice(device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
        for (size_t c = 0; c < g->plans.size() && e == cudaSuccess; ++c) {
            cudaStream_t sc = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking);
            if (e == cudaSuccess) g->side.push_back(sc);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) g->join.push_back(ev);
        }
        if (e != cudaSuccess) st = gfail(g, SRFMG_ECUDA, std::string("group streams: ") + cudaGetErrorString(e));
    }
    if (st != SRFMG_OK) {
        g_group_create_error = g->err;
        group_release(g);
        delete g;
        return st;
    }
    *out = g;
    return SRFMG_OK;
}

srfmg_status srfmg_group_solve(srfmg_group_handle g, const double *f, double *u, void *stream) {
    if (!g) return gfail(nullptr, SRFMG_EINVAL, "group handle is NULL");
    if (!f || !u) return gfail(g, SRFMG_EINVAL, "f and u must be device pointers");
    if (((uintptr_t)f & 15) || ((uintptr_t)u & 15)) return gfail(g, SRFMG_EINVAL, "f and u must be 16-byte aligned");
    if (overlap(f, g->total * sizeof(double), u, g->total * sizeof(double))) return gfail(g, SRFMG_EINVAL, "f and u overlap");
    NvtxRange range("srfmg_group_solve");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(g->device);
    if (e != cudaSuccess) return gfail(g, SRFMG_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    if (!g->use_graph) {
        e = group_enqueue(g, f, u, s);
        if (e != cudaSuccess) return gfail(g, SRFMG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    } else {
        if (!g->exec || g->gf != f || g->gu != u) {
            if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return gfail(g, SRFMG_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
            cudaError_t le = group_enqueue(g, f, u, g->cap);
            e = cudaStreamEndCapture(g->cap, &graph);
            if (le != cudaSuccess || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return gfail(g, SRFMG_ECUDA, std::string("group capture: ") + cudaGetErrorString(le != cudaSuccess ? le : e));
            }
            e = cudaGraphInstantiate(&g->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { g->exec = nullptr; return gfail(g, SRFMG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)); }
            g->gf = f;
            g->gu = u;
        }
        e = cudaGraphLaunch(g->exec, s);
        if (e != cudaSuccess) return gfail(g, SRFMG_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    }
    for (srfmg_plan *h : g->plans) h->solved = true;
    return SRFMG_OK;
}

srfmg_status srfmg_group_solve_host(srfmg_group_handle g, const double *f, double *u, void *stream) {
    if (!g) return gfail(nullptr, SRFMG_EINVAL, "group handle is NULL");
    if (!f || !u) return gfail(g, SRFMG_EINVAL, "f and u must be host pointers");
    NvtxRange range("srfmg_group_solve_host");
    cudaError_t e = cudaSetDevice(g->device);
    if (e == cudaSuccess && !g->f_stage) {
        e = cudaMalloc(&g->f_stage, g->total * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&g->u_stage, g->total * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (g->f_stage) cudaFree(g->f_stage);
            g->f_stage = nullptr;
            return gfail(g, SRFMG_ENOMEM, std::string("group staging buffers: ") + cudaGetErrorString(e));
        }
    }
    // every branch copies its own part in, solves it and copies it out, so
    // one size's copies overlap the others' kernels and copies
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaEventRecord(g->fork, s);
    for (size_t c = 0; c < g->plans.size() && e == cudaSuccess; ++c) {
        const size_t o = g->off[c], cells = (size_t)g->count[c] << g->m[c];
        cudaStream_t b = g->side[c];
        e = cudaStreamWaitEvent(b, g->fork, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->f_stage + o, f + o, cells * sizeof(double), cudaMemcpyHostToDevice, b);
        if (e == cudaSuccess)
            e = enqueue_all(g->plans[c], Io{g->f_stage + o, g->u_stage + o, nullptr, nullptr, nullptr}, b);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u + o, g->u_stage + o, cells * sizeof(double), cudaMemcpyDeviceToHost, b);
        if (e == cudaSuccess) e = cudaEventRecord(g->join[c], b);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g->join[c], 0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return gfail(g, SRFMG_ECUDA, std::string("group solve from host memory: ") + cudaGetErrorString(e));
    for (srfmg_plan *h : g->plans) h->solved = true;
    return SRFMG_OK;
}

srfmg_status srfmg_group_query(srfmg_group_handle g, int32_t *nplans, int64_t *total_cells) {
    if (!g) return gfail(nullptr, SRFMG_EINVAL, "group handle is NULL");
    if (nplans) *nplans = (int32_t)g->plans.size();
    if (total_cells) *total_cells = (int64_t)g->total;
    return SRFMG_OK;
}

srfmg_status srfmg_group_member(srfmg_group_handle g, int32_t i, srfmg_handle *plan, int32_t *log2_n,
                                int32_t *count, int64_t *offset) {
    if (!g) return gfail(nullptr, SRFMG_EINVAL, "group handle is NULL");
    if (i < 0 || i >= (int32_t)g->plans.size()) return gfail(g, SRFMG_EINVAL, "plan index out of range");
    if (plan) *plan = g->plans[i];
    if (log2_n) *log2_n = g->m[i];
    if (count) *count = g->count[i];
    if (offset) *offset = (int64_t)g->off[i];
    return SRFMG_OK;
}

srfmg_status srfmg_group_destroy(srfmg_group_handle g) {
    if (!g) return SRFMG_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    group_release(g);
    delete g;
    return SRFMG_OK;
}

const char *srfmg_group_last_error(srfmg_group_handle g) {
    return g ? g->err.c_str() : g_group_create_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free small solve.  The same one-block FMG kernel that
// srfmg_solve launches for N <= 2^12 without SR, with its coarsest-level
// inverse table in this static device array instead of plan memory from
// cudaMalloc.  In host code s_noalloc_ainv is only a host-side stand-in for
// the symbol: the device address comes from cudaGetSymbolAddress, once per
// device, with that device current.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double s_noalloc_ainv[SRFMG_NOALLOC_MAX_COARSE * SRFMG_NOALLOC_MAX_COARSE];

namespace {

constexpr int kNoallocMaxDevices = 64;

struct NoallocDevice {
    bool ready;        // symbol address looked up and smem limit raised
    double *ainv;      // device address of s_noalloc_ainv on this device
    int m0;            // log2_n_coarsest whose inverse the array holds (0: none)
};

NoallocDevice g_noalloc_dev[kNoallocMaxDevices];
std::mutex g_noalloc_mutex;
// host work arrays for the Gauss-Jordan inverse (static: no heap use)
long double g_noalloc_gj[SRFMG_NOALLOC_MAX_COARSE][2 * SRFMG_NOALLOC_MAX_COARSE];
double g_noalloc_inv[SRFMG_NOALLOC_MAX_COARSE * SRFMG_NOALLOC_MAX_COARSE];

// Same inverse as coarsest_inverse(), in static storage.
void noalloc_inverse(int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) g_noalloc_gj[i][j] = 0.0L;
    for (int i = 0; i < n; ++i) {
        g_noalloc_gj[i][i] = (i == 0 || i == n - 1) ? 3.0L : 2.0L;
        if (i > 0) g_noalloc_gj[i][i - 1] = -1.0L;
        if (i < n - 1) g_noalloc_gj[i][i + 1] = -1.0L;
        g_noalloc_gj[i][n + i] = 1.0L;
    }
    for (int c = 0; c < n; ++c) {
        long double piv = g_noalloc_gj[c][c];
        for (int j = 0; j < 2 * n; ++j) g_noalloc_gj[c][j] /= piv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            long double fct = g_noalloc_gj[r][c];
            if (fct == 0.0L) continue;
            for (int j = 0; j < 2 * n; ++j) g_noalloc_gj[r][j] -= fct * g_noalloc_gj[c][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) g_noalloc_inv[i * n + j] = (double)g_noalloc_gj[i][n + j];
}

}  // namespace

extern "C" srfmg_status srfmg_solve_small_noalloc(int32_t log2_n, int32_t log2_n_coarsest, int32_t nu1,
                                                  int32_t nu2, const double *f, double *u, void *stream) {
    if (log2_n_coarsest < 2 || log2_n_coarsest > 6 || log2_n <= log2_n_coarsest || log2_n > 12)
        return SRFMG_EINVAL;
    if (nu1 < 1 || nu1 > 4 || nu2 < 1 || nu2 > 4) return SRFMG_EINVAL;
    const size_t n = (size_t)1 << log2_n;
    if (!f || !u || ((uintptr_t)f & 15) || ((uintptr_t)u & 15)) return SRFMG_EINVAL;
    if ((const double *)u < f + n && f < (const double *)u + n) return SRFMG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SRFMG_ECUDA; }
    if (dev < 0 || dev >= kNoallocMaxDevices) return SRFMG_EUNSUPPORTED;

    // The lock is held through the launch: another host thread that changes
    // the uploaded coarsest level then does so only after this call's kernel
    // is enqueued (kernels of calls that overlap on the GPU still race).
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    double *ainv = nullptr;
    {
        NoallocDevice &d = g_noalloc_dev[dev];
        if (!d.ready) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, s_noalloc_ainv) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return SRFMG_ECUDA;
            }
            int optin = 0;
            if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
                cudaFuncSetAttribute(tail_kernel<kOpLaplace>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
                    cudaSuccess) {
                cudaGetLastError();
                return SRFMG_ECUDA;
            }
            d.ainv = (double *)ptr;
            d.m0 = 0;
            d.ready = true;
        }
        if (d.m0 != log2_n_coarsest) {
            const int n0 = 1 << log2_n_coarsest;
            noalloc_inverse(n0);
            if (cudaMemcpy(d.ainv, g_noalloc_inv, sizeof(double) * n0 * n0, cudaMemcpyHostToDevice) !=
                cudaSuccess) {
                cudaGetLastError();
                d.m0 = 0;
                return SRFMG_ECUDA;
            }
            d.m0 = log2_n_coarsest;
        }
        ainv = d.ainv;
    }
    TailArgs a;
    std::memset(&a, 0, sizeof(a));
    a.M0 = log2_n_coarsest;
    a.Mc = log2_n;
    a.nu1 = nu1;
    a.nu2 = nu2;
    a.mode = 0;
    a.g_in = f;
    a.g_exp = -2 * log2_n;
    a.u_out = u;
    a.Ainv = ainv;
    a.lam = 0.0;
    const size_t smem = tail_smem_doubles(log2_n_coarsest, log2_n) * sizeof(double);
    tail_kernel<kOpLaplace><<<1, kTailThreads, smem, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? SRFMG_OK : SRFMG_ECUDA;
}
