// srfmg_kernels.cuh -- sm_103a kernels of the FMG-FAS-SR solve (FP64 path).
//
// Notation: level l has n = 2^l cells; the solution u is stored unscaled, the
// right-hand side is stored scaled, g_l = h_l^2 rhs_l (h_l = 2^-l), so that
// the operator reads (h^2 L u)_i = F_{i-1/2} - F_{i+1/2} with the fluxes
// F_{i+1/2} = u_{i+1} - u_i and the odd ghost at the walls (F_{-1/2} = 2u_0,
// F_{n-1/2} = -2u_{n-1}), Sec. 4.  Scaling by powers of two is exact, so the
// scaled hierarchy is bit-identical to the unscaled one.
//
// FP64 runs at about 1/70 of the FP32 rate on this part, so every exact
// power-of-two scaling is done on the exponent bits with integer operations
// (scale2) instead of an FP64 multiply.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace srfmg {

// Terms of the Gauss-Seidel recurrence weighted below 2^-kTrunc are dropped;
// 2^-72 is far below the FP64 rounding of any value the recurrence produces.
constexpr int kTrunc = 72;

// Chunk length of the sweeps (one chunk per thread).  Odd, so that the threads
// of a warp, each reading its own chunk, touch distinct shared-memory banks
// (an even stride of 8-byte words serialises the warp); short, so that a
// block has many threads and each recurrence is a few dependent operations.
constexpr int kChunk = 9;

// Operators of the FP64 kernels (template parameter OP): -u'' = f, the
// variable-coefficient -(a u')' = f, and the Bratu problem -u'' + lam e^u = f.
constexpr int kOpLaplace = 0, kOpVarcoef = 1, kOpBratu = 2;
// The Bratu operator in the mixed precision (SRFMG_MIXED): the solution, the
// residual, the tau correction, the interpolations and the coarsest solve in
// FP64, the Newton Gauss-Seidel correction recurrence in FP32 (lex_sweep_nl_mx).
// (The mixed precision of the other two operators is the 64-bit fixed point of
// srfmg_fixed.cuh.)
constexpr int kOpBratuMx = 4;
__host__ __device__ constexpr bool op_vc(int op) { return op == kOpVarcoef; }
__host__ __device__ constexpr bool op_nl(int op) { return op == kOpBratu || op == kOpBratuMx; }

// Largest block of the level and segment kernels: one thread per chunk of at
// most 4224 + 2 cells (a segment) or 2944 cells (a tile).  Segment kernels
// are compiled for two such blocks per SM (at most 64 registers a thread).
constexpr int kSweepBlockMax = 512;

// Block size of the coarse tail: one sweep chunk per thread up to 2^12 cells.
constexpr int kTailBlock = 512;

// Programmatic dependent launch.  Every kernel of a solve starts with this:
// it waits until the preceding kernel in the stream has completed and its
// writes are visible, then allows the next kernel to begin launching, so
// that the next launch's set-up overlaps this kernel's work.  Both
// instructions do nothing for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Batched solves: a block serves problem blockIdx.y of the batch.  Every array
// of a level holds the problems one after another, so a pointer into an array
// of `cells` cells per problem moves by blockIdx.y * cells.  (The kernels keep
// the moved pointers in locals: writing a field of a kernel's parameter
// struct would make every thread copy the whole struct to local memory.)
template <typename T>
__device__ __forceinline__ T *batch_at(T *p, long long cells) {
    return p ? p + (long long)blockIdx.y * cells : p;
}

// Exact 2^k as a double, -1022 <= k <= 1023.
__device__ __forceinline__ double exp2i(int k) {
    return __longlong_as_double((long long)(1023 + k) << 52);
}

// x * 2^k by an exponent add (zero stays zero).  Valid for normal x whose
// result stays normal; the solver's values are many orders of magnitude away
// from the subnormal and overflow ranges.
__device__ __forceinline__ double scale2(double x, int k) {
    long long b = __double_as_longlong(x);
    long long inc = (b & 0x7ff0000000000000LL) ? ((long long)k << 52) : 0LL;
    return __longlong_as_double(b + inc);
}

// Coarse value with the odd reflection at the walls (u_{-1-j} = -u_j and
// u_{n+j} = -u_{n-1-j}); src[j - base] holds coarse cell j.
__device__ __forceinline__ double coarse_reflect(const double *src, int base, int j, int nc) {
    if (j < 0) return -src[-j - 1 - base];
    if (j >= nc) return -src[2 * nc - 1 - j - base];
    return src[j - base];
}

// Asynchronous staging of global memory into shared memory: cp.async copies of
// 8 bytes, issued by all threads of the block and all in flight at once, then
// one wait.  (A loop of plain loads would pay one L2 round trip per
// iteration.)
__device__ __forceinline__ void stage8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    size_t g = __cvta_generic_to_global(gmem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
}
// copy count 8-byte words src[0..count) to dst[0..count)
__device__ __forceinline__ void stage16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    size_t g = __cvta_generic_to_global(gmem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}
// copy count 8-byte words src[0..count) to dst[0..count): 16-byte copies when
// both addresses share their offset within 16 bytes (an odd first or last
// word by itself), 8-byte copies otherwise
__device__ __forceinline__ void stage_range(void *dst, const void *src, int count) {
    char *d = (char *)dst;
    const char *g = (const char *)src;
    if (count <= 0) return;
    if ((((uintptr_t)d ^ (uintptr_t)g) & 15) == 0) {
        const int head = ((uintptr_t)d & 15) ? 1 : 0;
        const int pairs = (count - head) >> 1;
        if (head && threadIdx.x == 0) stage8(d, g);
        for (int k = threadIdx.x; k < pairs; k += blockDim.x)
            stage16(d + 8 * head + 16 * (size_t)k, g + 8 * head + 16 * (size_t)k);
        if (((count - head) & 1) && threadIdx.x == blockDim.x - 1)
            stage8(d + 8 * (size_t)(count - 1), g + 8 * (size_t)(count - 1));
    } else {
        for (int k = threadIdx.x; k < count; k += blockDim.x) stage8(d + 8 * (size_t)k, g + 8 * (size_t)k);
    }
}
// wait for this thread's copies; follow with __syncthreads() before reading
__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Stage coarse cells [C0, C1) of a level of nc cells into c[0 .. C1-C0), with
// the odd reflection for the (at most two per side) ghost cells.  Two-phase:
// stage_coarse_async() issues the copies of the interior part;
// fill_coarse_ghosts() runs after the wait and a barrier.
template <typename T>
__device__ __forceinline__ void stage_coarse_async(T *c, const T *src, int C0, int C1, int nc) {
    const int j0 = max(C0, 0), j1 = min(C1, nc);
    stage_range(c + (j0 - C0), src + j0, j1 - j0);
}
template <typename T>
__device__ __forceinline__ void fill_coarse_ghosts(T *c, int C0, int C1, int nc) {
    for (int j = C0 + (int)threadIdx.x; j < C1; j += (int)blockDim.x) {
        if (j < 0) c[j - C0] = -c[(-j - 1) - C0];
        else if (j >= nc) c[j - C0] = -c[(2 * nc - 1 - j) - C0];
    }
}

// Fourth order FMG interpolation Pi (Sec. 4): the left child of J takes
// (-5, 35, 105, -7)/128 of coarse cells J-2..J+1, the right child the mirror.
// Written as u_J plus a combination of the coarse fluxes G_{j+1/2} = u_{j+1}-u_j
// (exact differences of nearby values), so the interpolated value carries a
// single rounding:  left  = u_J + (5G_{J-3/2} - 30G_{J-1/2} - 7G_{J+1/2})/128,
//                   right = u_J + (7G_{J-1/2} + 30G_{J+1/2} - 5G_{J+3/2})/128.
// Both children of J are formed together (they share the fluxes).
// c[j - cbase] must hold coarse cells J-2..J+2 (ghosts already reflected).
__device__ __forceinline__ void fmg_interp2(const double *c, int cbase, int J, double &left, double &right) {
    const double *p = c + (J - cbase);
    const double gm3 = p[-1] - p[-2], gm1 = p[0] - p[-1], gp1 = p[1] - p[0], gp3 = p[2] - p[1];
    const double sl = fma(5.0, gm3, fma(-30.0, gm1, -7.0 * gp1));
    const double sr = fma(7.0, gm1, fma(30.0, gp1, -5.0 * gp3));
    left = p[0] + scale2(sl, -7);
    right = p[0] + scale2(sr, -7);
}

// ---------------------------------------------------------------------------
// Lexicographic Gauss-Seidel sweep (omega = 1), in place, over the cells
// [lo, hi) of a level of n cells held in shared memory (u[i - base]; the
// neighbours lo-1 and hi are read and left unchanged; g[i - base]: scaled
// right-hand side over the same cells).
//
// Residual form.  With r_i = g_i - (F_{i-1/2} - F_{i+1/2}) the residual of the
// old values (flux form, odd ghost at the walls), the sweep adds
//   delta_i = (r_i + delta_{i-1}) / 2        (ascending; mirror descending)
// with delta = r/3 at the first wall cell and (r + delta_prev)/3 at the last
// wall cell (wall diagonal 3), and u_new = u_old + delta: one rounding per
// cell.  The correction entering the range (delta at lo-1) is zero: exact for
// a frozen patch neighbour, an approximation in a tile halo that is wider than
// the recurrence's memory.
//
// delta is a first-order linear recurrence with multiplier 1/2.  In sweep
// coordinates (q = i ascending, q = n-1-i descending) the cells are grouped in
// chunks of C consecutive positions aligned to the level, one chunk per thread
// (the number of chunks of [lo, hi) must not exceed blockDim.x).  Each chunk
// runs the recurrence from a zero carry with its cells in registers; the carry
// into a chunk is the fixed sum  sum_{j<=J} 2^(-jC) X_{c-1-j}  of the
// chunk-end values of the J+1 preceding chunks, J+1 = ceil(kTrunc / C), and
// the cell d places into its chunk's recurrence adds 2^-(d+1) times it.
// Terms weighted below 2^-kTrunc are dropped, so the result is the sequential
// sweep up to rounding.  With the fixed sum and level-aligned chunks, a cell's
// value depends only on the data of the (J+2)C cells before it, so two tiles
// that both hold a cell more than (J+2)C cells from their range start compute
// bitwise the same value: tiles agree exactly with their neighbours' halos,
// which keeps the tau correction consistent with the restricted solution at
// tile edges.
//
// Every chunk runs the same unrolled code: the loads go to in-range addresses
// (positions clamped to the staged cells) and cells outside [lo, hi) leave the
// recurrence unchanged, so no thread of a warp waits on a divergent path; the
// two wall cells are handled apart.  All threads of the block must call it.
// X holds one double per thread.
// ---------------------------------------------------------------------------
template <int C, bool PRELOAD, bool ASC>
__device__ __noinline__ void lex_sweep_dir(double *__restrict__ u, const double *__restrict__ g, int base,
                                              int lo, int hi, int n, double *X) {
    constexpr int s = ASC ? 1 : -1;                // sweep position q is u[a0 + s q]
    const int t = threadIdx.x;
    const int qlo = ASC ? lo : n - hi, qhi = ASC ? hi : n - lo;
    const int c_first = qlo / C, nch = (qhi - 1) / C - c_first + 1;
    const bool active = t < nch;
    const int q0 = (c_first + t) * C;
    // in-range cells [k0, k1) of the chunk; recurrence cells [ka, kb)
    const int k0 = max(qlo - q0, 0), k1 = min(qhi - q0, C);
    const bool wall0 = (q0 == 0) && (qlo == 0);      // sweep position 0 (a wall) is swept
    const bool wall1 = (q0 + k1 == n);               // sweep position n-1 (a wall) is swept
    const int ka = wall0 ? 1 : k0, kb = wall1 ? k1 - 1 : k1;
    const int qmin = max(qlo - 1, 0), qmax = min(qhi, n - 1);
    const int a0 = ASC ? -base : n - 1 - base;
    // a warp whose chunks are all full and away from the walls takes the
    // straight-line path (no clamps, no range selects)
    const bool fast = __all_sync(0xffffffffu, !active || (k0 == 0 && k1 == C && !wall0 && !wall1));
    double rr[C];
    double p = 0.0, r_end = 0.0;
    if (active) {
        double w[C + 2];   // u at positions q0-1 .. q0+C
        if (fast) {
            const double *up = u + (a0 + s * (q0 - 1)), *gp = g + (a0 + s * q0);
#pragma unroll
            for (int j = 0; j < C + 2; ++j) w[j] = up[s * j];
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const double r = gp[s * k] - ((w[k + 1] - w[k]) - (w[k + 2] - w[k + 1]));
                p = fma(0.5, p, scale2(r, -1));
                rr[k] = p;
            }
        } else {
#pragma unroll
            for (int j = 0; j < C + 2; ++j) w[j] = u[a0 + s * min(max(q0 - 1 + j, qmin), qmax)];
            if (wall0) p = (g[a0] - (scale2(w[1], 1) - (w[2] - w[1]))) * (1.0 / 3.0);
            if (wall1) {
                const double ue = u[a0 + s * (n - 1)], um = u[a0 + s * (n - 2)];
                r_end = g[a0 + s * (n - 1)] - ((ue - um) - (-scale2(ue, 1)));
            }
            double gv[C];
#pragma unroll
            for (int k = 0; k < C; ++k) gv[k] = g[a0 + s * min(max(q0 + k, qmin), qmax)];
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const double r = gv[k] - ((w[k + 1] - w[k]) - (w[k + 2] - w[k + 1]));
                const double pn = fma(0.5, p, scale2(r, -1));
                p = (k >= ka && k < kb) ? pn : p;
                rr[k] = p;
            }
        }
        X[t] = p;
    }
    __syncthreads();
    if (active) {
        constexpr int J = (kTrunc + C - 1) / C - 1;
        double cin = 0.0;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const int idx = t - 1 - j;
            const double x = X[max(idx, 0)];
            cin = fma(exp2i(-C), cin, idx >= 0 ? x : 0.0);
        }
        // PRELOAD: all loads first, then the arithmetic, then the stores (a
        // load after a store to a runtime-indexed address waits for the
        // store), for latency-bound blocks; otherwise the increments are
        // added in place, which needs fewer registers.
        if (fast) {
            double *up = u + (a0 + s * q0);
            double uo[C];
#pragma unroll
            for (int k = 0; k < C; ++k) uo[k] = PRELOAD ? up[s * k] : 0.0;
            double c = cin;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                c = scale2(c, -1);                   // 2^-(k+1) cin, exact
                if (PRELOAD) up[s * k] = uo[k] + (rr[k] + c);
                else up[s * k] += rr[k] + c;
            }
        } else {
            double uo[C];
#pragma unroll
            for (int k = 0; k < C; ++k) uo[k] = PRELOAD ? u[a0 + s * min(max(q0 + k, qmin), qmax)] : 0.0;
            const double ue = u[wall1 ? a0 + s * (n - 1) : a0 + s * min(max(q0, qmin), qmax)];   // in range
            double c = cin, dl = cin;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                if (k >= k0) c = scale2(c, -1);          // 2^-(k-k0+1) cin, exact
                dl = (k >= k0 && k < kb) ? rr[k] + c : dl;
                uo[k] += dl;
            }
#pragma unroll
            for (int k = 0; k < C; ++k)
                if (k >= k0 && k < kb) {
                    if (PRELOAD) u[a0 + s * (q0 + k)] = uo[k];
                    else u[a0 + s * (q0 + k)] += uo[k];
                }
            if (wall1) u[a0 + s * (n - 1)] = ue + (r_end + dl) * (1.0 / 3.0);
        }
    }
    __syncthreads();
}

template <int C, bool PRELOAD = false>
__device__ __forceinline__ void lex_sweep(double *__restrict__ u, const double *__restrict__ g, int base, int lo,
                                          int hi, int n, bool asc, double *X) {
    if (asc) lex_sweep_dir<C, PRELOAD, true>(u, g, base, lo, hi, n, X);
    else lex_sweep_dir<C, PRELOAD, false>(u, g, base, lo, hi, n, X);
}

// ---------------------------------------------------------------------------
// Nonlinear sweep for -u'' + lam e^u = f (pointwise Newton Gauss-Seidel, the
// nonlinear smoother S(L, u, f) of Fig. 1), in place, same layout and
// chunking as lex_sweep.  With e_i = cl e^{u_i} (cl = lam h^2 of the level,
// old values) one Newton step per cell gives the affine recurrence
//   delta_i = a_i (r_i + delta_{i-1}),  a_i = 1 / (2 + e_i)  (3 + e_i at a wall),
//   r_i = g_i - e_i - (F_{i-1/2} - F_{i+1/2})
// in the correction.  Each chunk runs it from a zero carry and publishes its
// end value X and the product Y of its a_i; the carry into a chunk is
// X_{c-1} + Y_{c-1} (X_{c-2} + Y_{c-2} (...)) over the J+1 = ceil(kTrunc / C)
// preceding chunks (every a_i <= 1/2, so the dropped terms are below 2^-72),
// and the cell d places into its chunk's recurrence adds (a_0 ... a_d) times it.
// X and Y hold one double per thread each.
// ---------------------------------------------------------------------------
template <int C, bool ASC>
__device__ __noinline__ void lex_sweep_nl_dir(double *__restrict__ u, const double *__restrict__ g, double cl,
                                              int base, int lo, int hi, int n, double *X, double *Y) {
    constexpr int s = ASC ? 1 : -1;
    const int t = threadIdx.x;
    const int qlo = ASC ? lo : n - hi, qhi = ASC ? hi : n - lo;
    const int c_first = qlo / C, nch = (qhi - 1) / C - c_first + 1;
    const bool active = t < nch;
    const int q0 = (c_first + t) * C;
    const int k0 = max(qlo - q0, 0), k1 = min(qhi - q0, C);
    const bool wall0 = (q0 == 0) && (qlo == 0);
    const bool wall1 = (q0 + k1 == n);
    const int ka = wall0 ? 1 : k0, kb = wall1 ? k1 - 1 : k1;
    const int qmin = max(qlo - 1, 0), qmax = min(qhi, n - 1);
    const int a0 = ASC ? -base : n - 1 - base;
    double rr[C], aa[C];
    double p = 0.0, A = 1.0, r_end = 0.0, a_end = 0.0;
    if (active) {
        double w[C + 2];
#pragma unroll
        for (int j = 0; j < C + 2; ++j) w[j] = u[a0 + s * min(max(q0 - 1 + j, qmin), qmax)];
        if (wall0) {
            const double e = cl * exp(w[1]);
            const double a = 1.0 / (3.0 + e);
            p = a * ((g[a0] - e) - (scale2(w[1], 1) - (w[2] - w[1])));
            A = a;
        }
        if (wall1) {
            const double ue = u[a0 + s * (n - 1)], um = u[a0 + s * (n - 2)];
            const double e = cl * exp(ue);
            r_end = (g[a0 + s * (n - 1)] - e) - ((ue - um) - (-scale2(ue, 1)));
            a_end = 1.0 / (3.0 + e);
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const double gv = g[a0 + s * min(max(q0 + k, qmin), qmax)];
            const double e = cl * exp(w[k + 1]);
            const double a = 1.0 / (2.0 + e);
            const double r = (gv - e) - ((w[k + 1] - w[k]) - (w[k + 2] - w[k + 1]));
            const bool in = k >= ka && k < kb;
            p = in ? a * (r + p) : p;
            A = in ? a * A : A;
            rr[k] = p;
            aa[k] = A;
        }
        X[t] = p;
        Y[t] = A;
    }
    __syncthreads();
    if (active) {
        constexpr int J = (kTrunc + C - 1) / C - 1;
        double cin = 0.0;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const int idx = t - 1 - j;
            const double x = X[max(idx, 0)], y = Y[max(idx, 0)];
            cin = idx >= 0 ? fma(y, cin, x) : 0.0;
        }
        double dl = cin;
#pragma unroll
        for (int k = 0; k < C; ++k)
            if (k >= k0 && k < kb) {
                dl = fma(aa[k], cin, rr[k]);
                u[a0 + s * (q0 + k)] += dl;
            }
        if (wall1) u[a0 + s * (n - 1)] += a_end * (r_end + dl);
    }
    __syncthreads();
}

template <int C>
__device__ __forceinline__ void lex_sweep_nl(double *__restrict__ u, const double *__restrict__ g, double cl,
                                             int base, int lo, int hi, int n, bool asc, double *X, double *Y) {
    if (asc) lex_sweep_nl_dir<C, true>(u, g, cl, base, lo, hi, n, X, Y);
    else lex_sweep_nl_dir<C, false>(u, g, cl, base, lo, hi, n, X, Y);
}

// ---------------------------------------------------------------------------
// Variable-coefficient sweep for -(a u')' = f (Gauss-Seidel, omega = 1), in
// place, same layout and chunking as lex_sweep.  With the face coefficients
// a_near (between the previous cell in sweep order and this one) and a_far
// (between this cell and the next), the update of a cell is
//   delta_q = (r_q + a_near delta_{q-1}) / (a_near + a_far),
//   r_q = g_q - (a_near (u_q - u_{q-1}) - a_far (u_{q+1} - u_q))
// (a wall face counts twice: odd ghost), an affine recurrence evaluated as in
// lex_sweep_nl with the multiplier a_near / (a_near + a_far).  For a
// coefficient that varies slowly between faces the multiplier stays near 1/2;
// the carry sum covers 11 chunks (99 cells), enough for multipliers up to 0.6
// (0.6^99 < 2^-72).  a[f - abase] is the coefficient of face f (faces f = 0..n,
// face f between cells f-1 and f); X and Y hold one double per thread.
// ---------------------------------------------------------------------------
constexpr int kTruncVc = 96;

template <int C, bool ASC>
__device__ __noinline__ void lex_sweep_vc_dir(double *__restrict__ u, const double *__restrict__ g,
                                              const double *__restrict__ a, int abase, int base, int lo, int hi,
                                              int n, double *X, double *Y) {
    constexpr int s = ASC ? 1 : -1;
    const int t = threadIdx.x;
    const int qlo = ASC ? lo : n - hi, qhi = ASC ? hi : n - lo;
    const int c_first = qlo / C, nch = (qhi - 1) / C - c_first + 1;
    const bool active = t < nch;
    const int q0 = (c_first + t) * C;
    const int k0 = max(qlo - q0, 0), k1 = min(qhi - q0, C);
    const bool wall0 = (q0 == 0) && (qlo == 0);
    const bool wall1 = (q0 + k1 == n);
    const int ka = wall0 ? 1 : k0, kb = wall1 ? k1 - 1 : k1;
    const int qmin = max(qlo - 1, 0), qmax = min(qhi, n - 1);
    const int a0 = ASC ? -base : n - 1 - base;
    // near face of sweep position q: face q ascending, face n - q descending;
    // the faces a chunk reads lie in [lo, hi] (clamped for the unused ones)
    const int fb0 = ASC ? 0 : n, fmin = lo, fmax = hi;
    double rr[C], aa[C];
    double p = 0.0, A = 1.0, r_end = 0.0, b_end = 0.0, al_end = 0.0;
    if (active) {
        double w[C + 2], an[C + 1];
#pragma unroll
        for (int j = 0; j < C + 2; ++j) w[j] = u[a0 + s * min(max(q0 - 1 + j, qmin), qmax)];
#pragma unroll
        for (int j = 0; j <= C; ++j) an[j] = a[min(max(fb0 + s * (q0 + j), fmin), fmax) - abase];
        if (wall0) {
            const double aw = an[0], af = an[1];
            const double D = scale2(aw, 1) + af;
            p = ((g[a0] - (aw * scale2(w[1], 1) - af * (w[2] - w[1])))) / D;
            A = 0.0;
        }
        if (wall1) {
            const int kw = k1 - 1;                      // the wall cell's place in the chunk
            const double ue = u[a0 + s * (n - 1)], um = u[a0 + s * (n - 2)];
            const double anr = a[fb0 + s * (n - 1) - abase], aw = a[fb0 + s * n - abase];
            const double D = anr + scale2(aw, 1);
            r_end = g[a0 + s * (n - 1)] - (anr * (ue - um) - aw * (-scale2(ue, 1)));
            b_end = 1.0 / D;
            al_end = anr * b_end;
            (void)kw;
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const double gv = g[a0 + s * min(max(q0 + k, qmin), qmax)];
            const double anr = an[k], afr = an[k + 1];
            const double b = 1.0 / (anr + afr);
            const double r = gv - (anr * (w[k + 1] - w[k]) - afr * (w[k + 2] - w[k + 1]));
            const bool in = k >= ka && k < kb;
            p = in ? fma(anr * b, p, r * b) : p;
            A = in ? (anr * b) * A : A;
            rr[k] = p;
            aa[k] = A;
        }
        X[t] = p;
        Y[t] = A;
    }
    __syncthreads();
    if (active) {
        constexpr int J = (kTruncVc + C - 1) / C - 1;
        double cin = 0.0;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const int idx = t - 1 - j;
            const double x = X[max(idx, 0)], y = Y[max(idx, 0)];
            cin = idx >= 0 ? fma(y, cin, x) : 0.0;
        }
        double dl = cin;
#pragma unroll
        for (int k = 0; k < C; ++k)
            if (k >= k0 && k < kb) {
                dl = fma(aa[k], cin, rr[k]);
                u[a0 + s * (q0 + k)] += dl;
            }
        if (wall1) u[a0 + s * (n - 1)] += fma(al_end, dl, b_end * r_end);
    }
    __syncthreads();
}

template <int C>
__device__ __forceinline__ void lex_sweep_vc(double *__restrict__ u, const double *__restrict__ g,
                                             const double *__restrict__ a, int abase, int base, int lo, int hi, int n,
                                             bool asc, double *X, double *Y) {
    if (asc) lex_sweep_vc_dir<C, true>(u, g, a, abase, base, lo, hi, n, X, Y);
    else lex_sweep_vc_dir<C, false>(u, g, a, abase, base, lo, hi, n, X, Y);
}

// ---------------------------------------------------------------------------
// Mixed-precision sweep (SRFMG_MIXED for the Bratu problem).  The split
// follows the precision roles of iterative refinement:
// the residual r of the old values is formed in FP64 (it decides what the
// smoother converges to), the correction recurrence that the Gauss-Seidel
// step solves for r runs in FP32 (it only decides how fast), and the
// correction is added to the FP64 solution.  GB300 issues FP64 at about 1/64
// of its FP32 rate, so the recurrence, the Newton denominator and the carry
// sums leave the FP64 pipe; the FP32 rounding of a correction (2^-24 of it)
// is far below the FP64 work it feeds, since the last corrections of a
// solve are of the size of its discretization error.  Layout, chunking and
// wall handling are those of lex_sweep_nl; X and Y hold one float per thread
// each (the caller's double arrays reinterpreted).  The carry covers fewer
// chunks than in FP64: terms weighted below 2^-33 are dropped (multipliers
// <= 1/2 over 36 cells).
// ---------------------------------------------------------------------------
constexpr int kTruncNlMx = 36;

// e^x for the mixed precision's Bratu terms, by Tang's table-driven method
// (P. T. P. Tang, ACM TOMS 15, 1989): x = (256 k + j) ln2/256 + r with
// |r| <= ln2/512 (plus rounding), e^x = 2^k 2^(j/256) e^r, e^r - 1 = r + r^2/2
// + r^3/6 (the dropped terms are below 1.5e-13 of the value).  The host fills
// g_exp2_tab[j] = 2^(j/256), j < 256, in long double and rounds once, and
// g_exp2_tab[256], [257] with ln2/256 split into a leading double and the
// rest (srfmg.cu, at the creation of a mixed Bratu plan).  About half of the
// FP64 operations of exp (slow on this part); relative error below 2e-13,
// checked against exp by srfmg_exp_error.  The residual's exponential enters
// the solution scaled by about lam / pi^2, far below the 1e-10 parity bound.
__device__ double g_exp2_tab[258];

__device__ __forceinline__ double exp_mx(double x) {
    if (!(fabs(x) <= 700.0)) return exp(x);          // (and inf, NaN)
    constexpr double kMagic = 6755399441055744.0;    // 1.5 * 2^52: adding it rounds to an integer
    constexpr double kInvL = 369.32993046757462751;  // 256 / ln 2
    const double sft = fma(x, kInvL, kMagic);
    const double nd = sft - kMagic;
    const int n = (int)(__double_as_longlong(sft) & 0xffffffffLL);
    double r = fma(-nd, __ldg(&g_exp2_tab[256]), x);
    r = fma(-nd, __ldg(&g_exp2_tab[257]), r);
    const double p = r * fma(r, fma(r, 1.0 / 6.0, 0.5), 1.0);
    const double T = __ldg(&g_exp2_tab[n & 255]);
    const double y = fma(T, p, T);
    return __longlong_as_double(__double_as_longlong(y) + ((long long)(n >> 8) << 52));
}

// Pointwise Newton Gauss-Seidel for -u'' + lam e^u = f, mixed: e_i = cl e^{u_i}
// and the residual r_i = g_i - e_i - (F_{i-1/2} - F_{i+1/2}) in FP64; the
// Newton denominator 2 + e_i (3 + e_i at a wall), its reciprocal and the
// recurrence delta_i = a_i (r_i + delta_{i-1}) in FP32.
template <int C, bool ASC>
__device__ __noinline__ void lex_sweep_nl_mx_dir(double *__restrict__ u, const double *__restrict__ g, double cl,
                                                 int base, int lo, int hi, int n, float *X, float *Y) {
    constexpr int s = ASC ? 1 : -1;
    const int t = threadIdx.x;
    const int qlo = ASC ? lo : n - hi, qhi = ASC ? hi : n - lo;
    const int c_first = qlo / C, nch = (qhi - 1) / C - c_first + 1;
    const bool active = t < nch;
    const int q0 = (c_first + t) * C;
    const int k0 = max(qlo - q0, 0), k1 = min(qhi - q0, C);
    const bool wall0 = (q0 == 0) && (qlo == 0);
    const bool wall1 = (q0 + k1 == n);
    const int ka = wall0 ? 1 : k0, kb = wall1 ? k1 - 1 : k1;
    const int qmin = max(qlo - 1, 0), qmax = min(qhi, n - 1);
    const int a0 = ASC ? -base : n - 1 - base;
    float rr[C], aa[C];
    float p = 0.0f, A = 1.0f, r_end = 0.0f, a_end = 0.0f;
    if (active) {
        double w[C + 2];
#pragma unroll
        for (int j = 0; j < C + 2; ++j) w[j] = u[a0 + s * min(max(q0 - 1 + j, qmin), qmax)];
        if (wall0) {
            const double e = cl * exp_mx(w[1]);
            const float a = __frcp_rn(3.0f + (float)e);
            p = a * (float)((g[a0] - e) - (scale2(w[1], 1) - (w[2] - w[1])));
            A = a;
        }
        if (wall1) {
            const double ue = u[a0 + s * (n - 1)], um = u[a0 + s * (n - 2)];
            const double e = cl * exp_mx(ue);
            r_end = (float)((g[a0 + s * (n - 1)] - e) - ((ue - um) - (-scale2(ue, 1))));
            a_end = __frcp_rn(3.0f + (float)e);
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const double gv = g[a0 + s * min(max(q0 + k, qmin), qmax)];
            const double e = cl * exp_mx(w[k + 1]);
            const float r = (float)((gv - e) - ((w[k + 1] - w[k]) - (w[k + 2] - w[k + 1])));
            const float a = __frcp_rn(2.0f + (float)e);
            const bool in = k >= ka && k < kb;
            p = in ? a * (r + p) : p;
            A = in ? a * A : A;
            rr[k] = p;
            aa[k] = A;
        }
        X[t] = p;
        Y[t] = A;
    }
    __syncthreads();
    if (active) {
        constexpr int J = (kTruncNlMx + C - 1) / C - 1;
        float cin = 0.0f;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const int idx = t - 1 - j;
            const float x = X[max(idx, 0)], y = Y[max(idx, 0)];
            cin = idx >= 0 ? fmaf(y, cin, x) : 0.0f;
        }
        float dl = cin;
#pragma unroll
        for (int k = 0; k < C; ++k)
            if (k >= k0 && k < kb) {
                dl = fmaf(aa[k], cin, rr[k]);
                u[a0 + s * (q0 + k)] += (double)dl;
            }
        if (wall1) u[a0 + s * (n - 1)] += (double)(a_end * (r_end + dl));
    }
    __syncthreads();
}

template <int C>
__device__ __forceinline__ void lex_sweep_nl_mx(double *__restrict__ u, const double *__restrict__ g, double cl,
                                                int base, int lo, int hi, int n, bool asc, double *X, double *Y) {
    float *Xf = reinterpret_cast<float *>(X), *Yf = reinterpret_cast<float *>(Y);
    if (asc) lex_sweep_nl_mx_dir<C, true>(u, g, cl, base, lo, hi, n, Xf, Yf);
    else lex_sweep_nl_mx_dir<C, false>(u, g, cl, base, lo, hi, n, Xf, Yf);
}

// One smoothing sweep of the operator OP (cl = lam h^2 of the level for the
// Bratu problem; a, abase: the face coefficients for the variable-coefficient
// problem; Y: a second per-thread array).
template <int OP, bool PRELOAD = false>
__device__ __forceinline__ void sweep_op(double *__restrict__ u, const double *__restrict__ g, double cl,
                                         const double *a, int abase, int base, int lo, int hi, int n, bool asc,
                                         double *X, double *Y) {
    if (OP == kOpBratu) lex_sweep_nl<kChunk>(u, g, cl, base, lo, hi, n, asc, X, Y);
    else if (OP == kOpBratuMx) lex_sweep_nl_mx<kChunk>(u, g, cl, base, lo, hi, n, asc, X, Y);
    else if (OP == kOpVarcoef) lex_sweep_vc<kChunk>(u, g, a, abase, base, lo, hi, n, asc, X, Y);
    else lex_sweep<kChunk, PRELOAD>(u, g, base, lo, hi, n, asc, X);
}

// Scaled tau-corrected coarse right-hand side at coarse cell J (Eqs. 6-7,
// Fig. 3 lines 3-5): g_{l-1,J} = 2(g_{2J} + g_{2J+1}) + (G_{J-1/2} - G_{J+1/2})
// - 2(F_{2J-1/2} - F_{2J+3/2}), where G are fluxes of uhat = R u on the coarse
// level and F fluxes of u; the value is h_{l-1}^2 times R rhs + L_{l-1} R u -
// R L_l u.  um1..up2 are u at fine cells 2J-2 .. 2J+3 (unused at a wall).
__device__ __forceinline__ double tau_rhs(double g0, double g1, double um2, double um1,
                                          double u0, double u1, double u2, double u3,
                                          int J, int nc) {
    double hJ = scale2(u0 + u1, -1);
    double Gl = (J == 0) ? scale2(hJ, 1) : hJ - scale2(um2 + um1, -1);
    double Gr = (J == nc - 1) ? -scale2(hJ, 1) : scale2(u2 + u3, -1) - hJ;
    double Fl = (J == 0) ? scale2(u0, 1) : u0 - um1;
    double Fr = (J == nc - 1) ? -scale2(u1, 1) : u2 - u1;
    double tau = (Gl - Gr) - scale2(Fl - Fr, 1);
    return scale2(g0 + g1, 1) + tau;
}

// Scaled tau-corrected coarse rhs for -(a u')' = f: as tau_rhs with every flux
// weighted by its face coefficient; the coarse faces J and J+1 are the fine
// faces 2J and 2J+2, whose coefficients a2J and a2J2 they take (injection).
__device__ __forceinline__ double tau_rhs_vc(double g0, double g1, double um2, double um1, double u0, double u1,
                                             double u2, double u3, int J, int nc, double a2J, double a2J2) {
    double hJ = scale2(u0 + u1, -1);
    double Gl = a2J * ((J == 0) ? scale2(hJ, 1) : hJ - scale2(um2 + um1, -1));
    double Gr = a2J2 * ((J == nc - 1) ? -scale2(hJ, 1) : scale2(u2 + u3, -1) - hJ);
    double Fl = a2J * ((J == 0) ? scale2(u0, 1) : u0 - um1);
    double Fr = a2J2 * ((J == nc - 1) ? -scale2(u1, 1) : u2 - u1);
    double tau = (Gl - Gr) - scale2(Fl - Fr, 1);
    return scale2(g0 + g1, 1) + tau;
}

// Coarsest level of -(a u')' = f: Thomas on h^2 L_a u = g (row i: -a_i u_{i-1}
// + (a_i + a_{i+1}) u_i - a_{i+1} u_{i+1}, a wall face counted twice), with
// the level's face coefficients a[0..n].  One thread; cp, dp hold n values.
__device__ void coarsest_thomas_vc(double *u, const double *g, int n, const double *a, double *cp, double *dp) {
    for (int i = 0; i < n; ++i) {
        const double al = (i == 0) ? scale2(a[0], 1) : a[i];
        const double ar = (i == n - 1) ? scale2(a[n], 1) : a[i + 1];
        const double diag = al + ar;
        const double lower = (i > 0) ? -a[i] : 0.0, upper = (i < n - 1) ? -a[i + 1] : 0.0;
        const double denom = (i > 0) ? diag - lower * cp[i - 1] : diag;
        cp[i] = upper / denom;
        dp[i] = ((i > 0) ? g[i] - lower * dp[i - 1] : g[i]) / denom;
    }
    u[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) u[i] = dp[i] - cp[i] * u[i + 1];
}

// The nonlinear part of the scaled tau rhs (Eqs. 1-2 with N = L + lam e^u):
// h_{l-1}^2 lam e^{uhat_J} - h_{l-1}^2 R(lam e^u)_J = cl (4 e^{uhat} - 2 (e^{u_2J} + e^{u_2J+1}))
// with cl = lam h_l^2 of the fine level and uhat = (u_2J + u_2J+1) / 2.  With
// u_2J = uhat + d, u_2J+1 = uhat - d this is -8 cl e^{uhat} sinh^2(d/2): one
// exponential instead of three, and no cancellation between terms of size
// 4 cl e^{uhat}.  For |d/2| < 2^-6 sinh(x)/x is its Taylor series to x^6 (the
// first dropped term is below 2^-66 of the value); otherwise the three
// exponentials.  MX: the mixed precision's exponential (exp_mx).
template <bool MX>
__device__ __forceinline__ double tau_nl(double cl, double u0, double u1) {
    auto E = [](double v) { return MX ? exp_mx(v) : exp(v); };
    const double uh = scale2(u0 + u1, -1);
    const double x = scale2(u0 - u1, -2);
    if (fabs(x) < 0.015625) {
        const double x2 = x * x;
        const double s = fma(x2, fma(x2, fma(x2, 1.0 / 5040.0, 1.0 / 120.0), 1.0 / 6.0), 1.0);
        return -8.0 * cl * E(uh) * (x2 * (s * s));
    }
    return cl * (4.0 * E(uh) - 2.0 * (E(u0) + E(u1)));
}

// ---------------------------------------------------------------------------
// K1: right-hand side hierarchy (appendix operator set-up): g on levels
// lin-1 .. lstop from level lin, g_{l-1,J} = 2 (g_{l,2J} + g_{l,2J+1}).
// Level lin is read from `in` scaled by 2^in_exp (f with in_exp = -2M).
// Each block reduces 2^depth consecutive cells of level lin in shared memory.
// ---------------------------------------------------------------------------
// Non-finite detection: kernels that read the caller's f (or form the
// functionals) OR kStatusNonFinite into the plan's status word, which the host
// reads with srfmg_check.  The exponent field 0x7ff marks inf and NaN.
constexpr int kStatusNonFinite = 1;
__device__ __forceinline__ bool nonfinite(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff;
}

struct RhsArgs {
    const double *in;
    int *status;               // non-finite f (when in is f)
    int in_exp;
    int lin, lstop, depth;
    int chunk_log;             // log2 of the cells each block reduces (>= depth)
    double *out[32];           // out[l] for the written levels
};

__global__ void rhs_hierarchy_kernel(RhsArgs a) {
    pdl_enter();
    extern __shared__ double sm[];
    const int chunk = 1 << a.chunk_log;       // cells of level lin per block (>= 2^depth)
    double *cur = sm, *nxt = sm + chunk;
    const long long base = (long long)blockIdx.x * chunk;
    const double *in = batch_at(a.in, 1LL << a.lin);
    stage_range(cur, in + base, chunk);
    stage_wait();
    __syncthreads();
    bool bad = false;
    if (a.in_exp)
        for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
            bad = bad || nonfinite(cur[i]);
            cur[i] = scale2(cur[i], a.in_exp);
        }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && a.status) atomicOr(a.status, kStatusNonFinite);
    int len = chunk;
    for (int l = a.lin; l > a.lstop && len > 1; --l) {
        const int half = len >> 1;
        double *dst = batch_at(a.out[l - 1], 1LL << (l - 1)) + (base >> (a.lin - l + 1));
        for (int J = threadIdx.x; J < half; J += blockDim.x) {
            double x = scale2(cur[2 * J] + cur[2 * J + 1], 1);
            nxt[J] = x;
            dst[J] = x;
        }
        __syncthreads();
        double *tmp = cur; cur = nxt; nxt = tmp;
        len = half;
    }
}

// ---------------------------------------------------------------------------
// Face coefficients of every level for -(a u')' = f from log a at the 2^M + 1
// faces of the finest level (NULL: a = 1): a_l[j] = exp(log_a[j 2^(M-l)]), the
// coarse faces taking the coefficient of the coinciding fine face.  out[l]
// holds 2^l + 1 values per problem (problem blockIdx.y).
//
// The kernel also sets *bad when the sweeps could not take the coefficient
// exactly: a log a that is not finite or lies beyond +-700 (a would overflow or
// vanish), or two adjacent faces of a level of 2^7 cells or more whose
// coefficients differ by more than a factor 1.5.  The variable-coefficient
// sweep carries over 99 cells, which is exact to 2^-72 for multipliers
// a_near / (a_near + a_far) <= 0.6, i.e. for a contrast of at most 1.5
// between neighbouring faces; levels of at most 64 cells carry over the whole
// level and need no bound.
// ---------------------------------------------------------------------------
struct CoefArgs {
    const double *log_a;
    int M, M0;
    int *bad;
    double *out[32];
};

constexpr int kCoefCheckLevel = 7;
constexpr double kLogContrastMax = 0.405465108108164382;   // ln 1.5
constexpr double kLogAMax = 700.0;

__global__ void coef_hierarchy_kernel(CoefArgs a) {
    pdl_enter();
    const long long nf = (1LL << a.M) + 1;
    const double *la = batch_at(a.log_a, nf);
    bool ok = true;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nf; j += (long long)gridDim.x * blockDim.x) {
        const double lv = la ? la[j] : 0.0;
        const double v = la ? exp(lv) : 1.0;
        ok = ok && fabs(lv) <= kLogAMax;                 // false for NaN
        for (int l = a.M; l >= a.M0; --l) {
            const int sh = a.M - l;
            if (j & ((1LL << sh) - 1)) break;
            batch_at(a.out[l], (1LL << l) + 1)[j >> sh] = v;
            const long long jn = j + (1LL << sh);        // the next face of level l
            if (la && l >= kCoefCheckLevel && jn < nf)
                ok = ok && fabs(la[jn] - lv) <= kLogContrastMax;
        }
    }
    if (!ok) atomicOr(a.bad, 1);
}

// ---------------------------------------------------------------------------
// dL/dlog a at the 2^M + 1 faces of the finest level from the solution u and
// the adjoint state lam = A^{-1} dL/du of -(a u')' = f (the derivative of the
// variable-coefficient operator): face f, between cells f-1 and f, carries the
// flux a_f (u_f - u_{f-1}) n^2 into cell f (+) and cell f-1 (-), so
//   dL/dlog a_f = -a_f (u_f - u_{f-1}) (lam_f - lam_{f-1}) n^2,
// and the wall faces, through the odd ghost, -a (2 u) lam n^2 with their one
// cell.  One thread per face (grid-stride), problem blockIdx.y.
// ---------------------------------------------------------------------------
__global__ void coef_gradient_kernel(const double *__restrict__ u, const double *__restrict__ lam,
                                     const double *__restrict__ a, double *__restrict__ out, int M) {
    pdl_enter();
    const long long n = 1LL << M;
    const double n2 = (double)n * (double)n;
    const double *up = batch_at(u, n), *lp = batch_at(lam, n), *ap = batch_at(a, n + 1);
    double *op = batch_at(out, n + 1);
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f <= n; f += (long long)gridDim.x * blockDim.x) {
        double du, dl;
        if (f == 0) {
            du = 2.0 * up[0];
            dl = lp[0];
        } else if (f == n) {
            du = 2.0 * up[n - 1];
            dl = lp[n - 1];
        } else {
            du = up[f] - up[f - 1];
            dl = lp[f] - lp[f - 1];
        }
        op[f] = -(ap[f] * du * dl) * n2;
    }
}

// ---------------------------------------------------------------------------
// Stored-level passes (global lexicographic smoothing).  A block owns the
// tile [s, s+T) of level l and loads it with a halo of H cells per side; the
// halo is wider than the Gauss-Seidel carry horizon, so the tile's values are
// those of the sequential sweep over the whole level (Sec. 4: "subdomain
// solver applied to the entire grid").
// ---------------------------------------------------------------------------
struct LevelArgs {
    int l, n, tile, halo, nu;
    int maxlen, maxc, maxch;   // shared-memory layout sizes (doubles)
    const double *u_src;       // level l iterate, or level l-1 for the FMG interpolation
    const double *g;           // g_l, or f when g_exp != 0 (scaled by 2^g_exp on load)
    int g_exp;
    const double *uc_src;      // up pass: corrected level l-1
    double *u_out;             // level l after the pass (tile)
    double *uc_out;            // down pass: restricted solution on level l-1
    double *gc_out;            // down pass: tau-corrected g_{l-1}
    double lam;                // Bratu: lam of -u'' + lam e^u = f (0 otherwise)
    const double *coef;        // variable coefficient: face coefficients of level l (2^l + 1)
};

// Shared-memory layout of one stored-level block (the host reserves
// 2 maxlen + 2 maxc + maxch doubles; this path uses the first
// 2 maxlen + maxc + maxch).
struct LevelSmem {
    double *u, *g, *c, *X, *Y;   // Y: second carry array of the nonlinear sweeps
    double *a;                // variable coefficient: faces [L0, L1] (the host adds maxlen words)
    int L0, L1, C0, C1;       // fine range [L0,L1), coarse range [C0,C1)
};

__device__ __forceinline__ LevelSmem level_smem(double *sm, int s, int T, int H, int n, int maxlen, int maxc,
                                                int maxch) {
    LevelSmem m;
    m.L0 = max(0, s - H);
    m.L1 = min(n, s + T + H);
    m.C0 = (m.L0 >> 1) - 2;
    m.C1 = ((m.L1 - 1) >> 1) + 3;
    m.u = sm;
    m.g = m.u + maxlen;
    m.c = m.g + maxlen;
    m.X = m.c + maxc;
    m.Y = m.X + maxch;
    m.a = m.c + 2 * maxc;     // past the whole X/Y region (maxc words)
    return m;
}

// Smoothing of a loaded range by nu sweeps in place, ascending first and
// reversed after every sweep (appendix "symmetrize").  The swept range
// shrinks by one cell per sweep on each side that is not a wall, so that
// every sweep reads neighbours the previous one wrote.
template <int OP>
__device__ void smooth_range(LevelSmem &m, int n, int nu, double cl) {
    int lo = (m.L0 == 0) ? 0 : m.L0 + 1;
    int hi = (m.L1 == n) ? n : m.L1 - 1;
    for (int k = 0; k < nu; ++k) {
        sweep_op<OP>(m.u, m.g, cl, m.a, m.L0, m.L0, lo, hi, n, (k & 1) == 0, m.X, m.Y);
        if (lo > 0) ++lo;
        if (hi < n) --hi;
    }
}

template <bool FROM_PI, int OP>
__global__ void __launch_bounds__(kSweepBlockMax, 2) level_down_kernel(LevelArgs a) {
    pdl_enter();
    extern __shared__ double sm[];
    const int s = blockIdx.x * a.tile;
    const int n = a.n, nc = n >> 1;
    const double *u_src = batch_at(a.u_src, FROM_PI ? nc : n), *g = batch_at(a.g, n);
    double *u_out = batch_at(a.u_out, n), *uc_out = batch_at(a.uc_out, nc), *gc_out = batch_at(a.gc_out, nc);
    LevelSmem m = level_smem(sm, s, a.tile, a.halo, n, a.maxlen, a.maxc, a.maxch);
    if (op_vc(OP)) stage_range(m.a, batch_at(a.coef, n + 1) + m.L0, m.L1 - m.L0 + 1);
    stage_range(m.g, g + m.L0, m.L1 - m.L0);
    if (FROM_PI) stage_coarse_async(m.c, u_src, m.C0, m.C1, nc);
    else stage_range(m.u, u_src + m.L0, m.L1 - m.L0);
    stage_wait();
    __syncthreads();
    if (a.g_exp)
        for (int i = m.L0 + (int)threadIdx.x; i < m.L1; i += (int)blockDim.x)
            m.g[i - m.L0] = scale2(m.g[i - m.L0], a.g_exp);
    if (FROM_PI) {
        fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
        __syncthreads();
        for (int J = (m.L0 >> 1) + (int)threadIdx.x; J < (m.L1 >> 1); J += (int)blockDim.x)
            fmg_interp2(m.c, m.C0, J, m.u[2 * J - m.L0], m.u[2 * J + 1 - m.L0]);
    }
    __syncthreads();
    const double cl = scale2(a.lam, -2 * a.l);       // lam h_l^2
    smooth_range<OP>(m, n, a.nu, cl);
    const double *u = m.u;
    // restriction of the solution and tau-corrected coarse rhs of the tile
    for (int J = (s >> 1) + threadIdx.x; J < ((s + a.tile) >> 1); J += blockDim.x) {
        int i0 = 2 * J - m.L0;
        double um2 = (J > 0) ? u[i0 - 2] : 0.0, um1 = (J > 0) ? u[i0 - 1] : 0.0;
        double u2 = (J < nc - 1) ? u[i0 + 2] : 0.0, u3 = (J < nc - 1) ? u[i0 + 3] : 0.0;
        uc_out[J] = scale2(u[i0] + u[i0 + 1], -1);
        double gc = (op_vc(OP))
                        ? tau_rhs_vc(m.g[i0], m.g[i0 + 1], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, m.a[i0],
                                     m.a[i0 + 2])
                        : tau_rhs(m.g[i0], m.g[i0 + 1], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc);
        if (op_nl(OP)) gc += tau_nl<OP == kOpBratuMx>(cl, u[i0], u[i0 + 1]);
        gc_out[J] = gc;
    }
    for (int i = s + threadIdx.x; i < s + a.tile; i += blockDim.x) u_out[i] = u[i - m.L0];
}

// Up pass (Eq. 4): u_l += P (u_{l-1} - R u_l), then nu sweeps.
template <int OP>
__global__ void __launch_bounds__(kSweepBlockMax, 2) level_up_kernel(LevelArgs a) {
    pdl_enter();
    extern __shared__ double sm[];
    const int s = blockIdx.x * a.tile;
    const int n = a.n, nc = n >> 1;
    const double *u_src = batch_at(a.u_src, n), *g = batch_at(a.g, n), *uc_src = batch_at(a.uc_src, nc);
    double *u_out = batch_at(a.u_out, n);
    LevelSmem m = level_smem(sm, s, a.tile, a.halo, n, a.maxlen, a.maxc, a.maxch);
    if (op_vc(OP)) stage_range(m.a, batch_at(a.coef, n + 1) + m.L0, m.L1 - m.L0 + 1);
    stage_range(m.g, g + m.L0, m.L1 - m.L0);
    stage_range(m.u, u_src + m.L0, m.L1 - m.L0);
    stage_coarse_async(m.c, uc_src, m.C0, m.C1, nc);
    stage_wait();
    __syncthreads();
    if (a.g_exp)
        for (int i = m.L0 + (int)threadIdx.x; i < m.L1; i += (int)blockDim.x)
            m.g[i - m.L0] = scale2(m.g[i - m.L0], a.g_exp);
    // coarse correction c_J = u_{l-1,J} - (R u_l)_J from the staged tile.  The
    // coarse cells whose children lie outside it (at most two per tile end,
    // never at a wall) get no correction: they only reach the frozen end cells
    // L0 and L1-1, whose difference dies out inside the halo.
    for (int j = max(m.C0, 0) + (int)threadIdx.x; j < min(m.C1, nc); j += (int)blockDim.x) {
        const int i0 = 2 * j;
        const bool inside = i0 >= m.L0 && i0 + 1 < m.L1;
        m.c[j - m.C0] = inside ? m.c[j - m.C0] - scale2(m.u[i0 - m.L0] + m.u[i0 + 1 - m.L0], -1) : 0.0;
    }
    __syncthreads();
    fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
    __syncthreads();
    // second order prolongation: child = 3/4 parent + 1/4 neighbour on its side
    for (int i = m.L0 + (int)threadIdx.x; i < m.L1; i += (int)blockDim.x) {
        int J = i >> 1, nb = (i & 1) ? J + 1 : J - 1;
        double corr = scale2(fma(3.0, m.c[J - m.C0], m.c[nb - m.C0]), -2);
        m.u[i - m.L0] += corr;
    }
    __syncthreads();
    smooth_range<OP>(m, n, a.nu, scale2(a.lam, -2 * a.l));
    const double *u = m.u;
    for (int i = s + threadIdx.x; i < s + a.tile; i += blockDim.x) u_out[i] = u[i - m.L0];
}

// ---------------------------------------------------------------------------
// SR level (Fig. 3): one block per segment [s, s+W) with extended patch
// E = [s-b, s+W+b) clipped to the domain and one frozen cell on each side.
// The fine level exists only in shared memory.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Functionals of the fine-grid solution, collected while the segments are swept
// (Fig. 3 computes a functional of the fine grid in the post-smoothing leg; the
// paper's closing section names such functionals as one way to get quantities
// of interest out of a solution that is never stored).  Per problem:
//   F0 = h sum u_i, F1 = h sum u_i^2, F2 = max |u_i|,
//   F3 = h sum (u_i - r_i)^2, F4 = max |u_i - r_i|  (r a reference; 0 without one).
// Each post-leg block reduces its segment interior into kNumFunc partials in a
// fixed order, and functionals_finish_kernel reduces the segments in a fixed
// order, so a solve gives the same bits on every run.
// ---------------------------------------------------------------------------
constexpr int kNumFunc = 5;
constexpr int kFinishThreads = 1024;

struct FuncAcc {
    double v[kNumFunc];
    __device__ FuncAcc() {
#pragma unroll
        for (int k = 0; k < kNumFunc; ++k) v[k] = 0.0;
    }
    __device__ __forceinline__ void add(double x, const double *ref, long long i) {
        v[0] += x;
        v[1] = fma(x, x, v[1]);
        v[2] = fmax(v[2], fabs(x));
        if (ref) {
            const double d = x - ref[i];
            v[3] = fma(d, d, v[3]);
            v[4] = fmax(v[4], fabs(d));
        }
    }
    __device__ __forceinline__ void merge(const double *e) {
        v[0] += e[0];
        v[1] += e[1];
        v[2] = fmax(v[2], e[2]);
        v[3] += e[3];
        v[4] = fmax(v[4], e[4]);
    }
};

// The reductions below keep FP64 instructions out of the shuffle trees: an FP64
// warp instruction occupies this GPU's narrow FP64 pipe for many cycles, and a
// butterfly over five values in every warp of every segment block cost more
// than the post-leg itself.
//
// Maximum over the warp of non-negative doubles (or NaN) by their bit patterns,
// which order like the values; NaN (above every finite value and inf) wins.
__device__ __forceinline__ double warp_max_nonneg(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
    }
    return __longlong_as_double((long long)b);
}

// round(x 2^k) of the bits b of a double, for |x| 2^k < 2^60 (zero and
// subnormals give 0).
__device__ __forceinline__ long long round_scaled_bits(long long b, int k) {
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = e - 1075 + k;
    long long v;
    if (sh >= 0) v = m << sh;
    else if (sh > -63) v = (m + (1LL << (-sh - 1))) >> (-sh);
    else v = 0;
    return b < 0 ? -v : v;
}

// Sum over the warp: every lane's value on the integer grid 2^-k of the warp's
// largest exponent (|v| < 2^56, so the 32-lane sum stays below 2^61), summed
// exactly, one conversion back.  The rounding moves each term by at most
// 2^-56 of the largest; the result (in every lane) does not depend on which
// lane holds which term's neighbours.  A non-finite lane takes FP64 sums.
__device__ __forceinline__ double warp_sum(double x) {
    const long long b = __double_as_longlong(x);
    const unsigned emax = __reduce_max_sync(0xffffffffu, (unsigned)((b >> 52) & 0x7ff));
    if (emax == 0x7ff) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
    }
    const int k = 1078 - (int)emax;                 // |x| < 2^(emax - 1022)
    long long v = round_scaled_bits(b, k);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v == 0 ? 0.0 : scale2((double)v, -k);
}

// Reduce the block's accumulators (sums F0, F1, F3; maxima F2, F4) in a fixed
// order; the result is valid in thread 0.  blockDim.x is a multiple of 32, at
// most 1024, and every thread of the block calls it once.
__device__ __forceinline__ void func_block_reduce(FuncAcc &q) {
    __shared__ double red[kNumFunc][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kNumFunc; ++k) {
        const double x = (k == 2 || k == 4) ? warp_max_nonneg(q.v[k]) : warp_sum(q.v[k]);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < kNumFunc; ++k) {
            const double x = lane < nw ? red[k][lane] : 0.0;
            q.v[k] = (k == 2 || k == 4) ? warp_max_nonneg(x) : warp_sum(x);
        }
    }
}

// Segment partials (nseg per problem, problem blockIdx.y) -> out[kNumFunc] per
// problem; one block of kFinishThreads threads per problem (a few segments per
// thread, so the chain of dependent loads and adds stays short).
__global__ void __launch_bounds__(kFinishThreads) functionals_finish_kernel(const double *fpart, int nseg, int M,
                                                                        double *out, int *status) {
    pdl_enter();
    const double *src = batch_at(fpart, (long long)nseg * kNumFunc);
    FuncAcc q;
    for (int j = threadIdx.x; j < nseg; j += blockDim.x) q.merge(src + (long long)j * kNumFunc);
    func_block_reduce(q);
    if (threadIdx.x == 0) {
        const double h = scale2(1.0, -M);
        double *o = batch_at(out, kNumFunc);
        o[0] = q.v[0] * h;
        o[1] = q.v[1] * h;
        o[2] = q.v[2];
        o[3] = q.v[3] * h;
        o[4] = q.v[4];
        bool bad = false;
#pragma unroll
        for (int k = 0; k < kNumFunc; ++k) bad = bad || nonfinite(o[k]);
        if (bad && status) atomicOr(status, kStatusNonFinite);
    }
}

struct SegArgs {
    int M, n, W, b, nu;
    int maxlen, maxc, maxch;   // shared-memory layout sizes (doubles)
    int seg0;                  // post-leg: first segment (block x handles segment seg0 + x)
    int local_tau;             // pre-leg: tau of the edge coarse cells from the own patch (no seam pass)
    const double *f;           // right-hand side, unscaled (the finest level)
    const double *g_in;        // SR level below the finest: its scaled rhs g_M (then f is unused)
    const double *u_in;        // pre-leg of an SR level below the top: its assembled iterate (no Pi)
    const double *uc_src;      // level M-1
    double *uc_out;            // pre-leg: restricted solution on level M-1
    double *gc_out;            // pre-leg: tau-corrected g_{M-1}
    double *seam;              // pre-leg: 6 fine values per segment
    double *u_out;             // post-leg: the solution of segments seg0.. (NULL: not written)
    const double *u_ref;       // post-leg: reference for the functionals (NULL: none)
    double *fpart;             // post-leg: kNumFunc partials per segment (NULL: no functionals)
    double lam;                // Bratu: lam (0 otherwise)
    const double *coef;        // variable coefficient: face coefficients of level M (2^M + 1)
    // post-leg option FAS recompute (the correction of Eq. 4 on the recomputed
    // pre-smoothed segment): the pre-leg keeps the level M-1 iterate it
    // interpolates (its segment's coarse cells) and the first and last b + 1
    // pre-smoothed interior cells of its segment; the post-leg (uc_corr set)
    // interpolates uc_src = that iterate, smooths nu_pre times as the pre-leg did,
    // takes its buffer and frozen cells from the neighbours' kept cells, adds
    // P (uc_corr - uhat) and smooths nu times without Kaczmarz
    double *u_old_out, *edge_out;
    const double *uc_corr, *uhat, *edge_in;
    int nu_pre;
    int c2_off;                // FP64 post-leg recompute: offset (doubles) of a second coarse array
};

// (the host reserves 2 maxlen + 2 maxc + maxch doubles; this path uses the
// first 2 maxlen + maxc + maxch)
struct SegSmem {
    double *u, *g, *c, *X, *Y;
    double *a;                 // variable coefficient: faces [lo, hi]
    int e0, e1, lo, hi, C0, C1;
};

__device__ __forceinline__ SegSmem seg_smem(double *sm, const SegArgs &a, int s) {
    SegSmem m;
    m.e0 = max(0, s - a.b);
    m.e1 = min(a.n, s + a.W + a.b);
    m.lo = (m.e0 > 0) ? m.e0 - 1 : 0;
    m.hi = (m.e1 < a.n) ? m.e1 + 1 : a.n;
    m.C0 = (m.lo >> 1) - 2;
    m.C1 = ((m.hi - 1) >> 1) + 3;
    m.u = sm;
    m.g = m.u + a.maxlen;
    m.c = m.g + a.maxlen;
    m.X = m.c + a.maxc;
    m.Y = m.X + a.maxch;
    m.a = m.c + 2 * a.maxc;
    return m;
}

// Load the patch [lo, hi) (patch and frozen cells) of an SR level M: the
// iterate Pi u_{M-1} (or, with u_in, the assembled iterate of a level below
// the top, in the down leg) and the scaled rhs (f 2^-2M on the finest level,
// g_in on the levels below it).
__device__ void seg_load(SegSmem &m, const SegArgs &a) {
    const int nc = a.n >> 1;
    if (a.u_in) stage_range(m.u, batch_at(a.u_in, a.n) + m.lo, m.hi - m.lo);
    else stage_coarse_async(m.c, batch_at(a.uc_src, nc), m.C0, m.C1, nc);
    if (a.g_in) stage_range(m.g, batch_at(a.g_in, a.n) + m.lo, m.hi - m.lo);
    else stage_range(m.g, batch_at(a.f, a.n) + m.lo, m.hi - m.lo);
    if (a.coef) stage_range(m.a, batch_at(a.coef, a.n + 1) + m.lo, m.hi - m.lo + 1);
    stage_wait();
    __syncthreads();
    if (!a.g_in)
        for (int i = m.lo + (int)threadIdx.x; i < m.hi; i += (int)blockDim.x)
            m.g[i - m.lo] = scale2(m.g[i - m.lo], -2 * a.M);
    if (a.u_in) {
        __syncthreads();
        return;
    }
    fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
    __syncthreads();
    for (int J = (m.lo >> 1) + (int)threadIdx.x; 2 * J < m.hi; J += (int)blockDim.x) {
        double l, r;
        fmg_interp2(m.c, m.C0, J, l, r);
        if (2 * J >= m.lo) m.u[2 * J - m.lo] = l;
        if (2 * J + 1 < m.hi) m.u[2 * J + 1 - m.lo] = r;
    }
    __syncthreads();
}

// K5: pre-smoothing leg of the SR level (Fig. 3 lines 1-5): Pi, nu1 sweeps on
// the extended patch, restricted solution on the segment's coarse cells, tau
// rhs on the coarse cells whose stencil lies in the segment, seam values for
// the two edge cells (formed from the assembled level by seam_tau_kernel);
// with local_tau the edge cells' tau too, from the patch's own buffer cells
// (Fig. 3 line 4 read literally; b >= 2 keeps their stencil in the patch).
template <int OP>
__global__ void __launch_bounds__(kSweepBlockMax, 2) sr_pre_kernel(SegArgs a) {
    pdl_enter();
    extern __shared__ double sm[];
    const int s = blockIdx.x * a.W;
    const int n = a.n, nc = n >> 1;
    SegSmem m = seg_smem(sm, a, s);
    seg_load(m, a);
    const int J0 = s >> 1, J1 = (s + a.W) >> 1;
    if (a.u_old_out) {        // the interpolated iterate on the segment's coarse cells (post-leg recompute)
        double *uo = batch_at(a.u_old_out, nc);
        for (int J = J0 + (int)threadIdx.x; J < J1; J += (int)blockDim.x) uo[J] = m.c[J - m.C0];
    }
    const double cl = scale2(a.lam, -2 * a.M);
    for (int k = 0; k < a.nu; ++k)
        sweep_op<OP>(m.u, m.g, cl, m.a, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y);
    const double *u = m.u;
    if (a.edge_out) {         // the pre-smoothed interior cells the neighbours' patches read
        const int ne = a.b + 1;
        double *eo = batch_at(a.edge_out, (long long)(n / a.W) * 2 * ne) + (size_t)blockIdx.x * 2 * ne;
        for (int k = threadIdx.x; k < ne; k += blockDim.x) {
            eo[k] = u[s + k - m.lo];
            eo[ne + k] = u[s + a.W - ne + k - m.lo];
        }
    }
    double *uc_out = batch_at(a.uc_out, nc), *gc_out = batch_at(a.gc_out, nc);
    for (int J = J0 + threadIdx.x; J < J1; J += blockDim.x) {
        int i0 = 2 * J - m.lo;
        uc_out[J] = scale2(u[i0] + u[i0 + 1], -1);
        bool edge = !a.local_tau && ((J == J0 && J > 0) || (J == J1 - 1 && J < nc - 1));
        if (!edge) {
            double um2 = (J > 0) ? u[i0 - 2] : 0.0, um1 = (J > 0) ? u[i0 - 1] : 0.0;
            double u2 = (J < nc - 1) ? u[i0 + 2] : 0.0, u3 = (J < nc - 1) ? u[i0 + 3] : 0.0;
            double gc = (op_vc(OP))
                            ? tau_rhs_vc(m.g[i0], m.g[i0 + 1], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, m.a[i0],
                                         m.a[i0 + 2])
                            : tau_rhs(m.g[i0], m.g[i0 + 1], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc);
            if (op_nl(OP)) gc += tau_nl<OP == kOpBratuMx>(cl, u[i0], u[i0 + 1]);
            gc_out[J] = gc;
        }
    }
    if (threadIdx.x < 6) {
        int k = threadIdx.x;
        int i = (k < 3) ? s + k : s + a.W - 6 + k;
        batch_at(a.seam, 6LL * (a.n / a.W))[(size_t)blockIdx.x * 6 + k] = u[i - m.lo];
    }
}

// tau rhs of the two coarse cells at each interior segment boundary, from the
// assembled fine values (seams) and the restricted solution (appendix down
// leg).  Thread k handles the boundary s = (k+1) W.
template <int OP>
__global__ void seam_tau_kernel(SegArgs a, int nseg) {
    pdl_enter();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nseg - 1) return;
    const double *seam = batch_at(a.seam, 6LL * nseg);
    // restricted rhs R g of the coarse cell J' from the level's rhs (f 2^-2M, or g_in)
    const double *rf = a.g_in ? batch_at(a.g_in, a.n) : batch_at(a.f, a.n);
    const int rexp = a.g_in ? 1 : 1 - 2 * a.M;
    double *uc_out = batch_at(a.uc_out, a.n / 2), *gc_out = batch_at(a.gc_out, a.n / 2);
    const int s = (k + 1) * a.W;
    const double *L = seam + (size_t)k * 6, *R = seam + (size_t)(k + 1) * 6;
    // fine cells s-3 .. s+2 of the assembled level
    double f3 = L[3], f2 = L[4], f1 = L[5], p0 = R[0], p1 = R[1], p2 = R[2];
    const int J = (s >> 1) - 1;         // last coarse cell of the left segment
    // coarse fluxes G from the restricted solution, fine fluxes F from the seams
    const double hm1 = uc_out[J - 1], h0 = uc_out[J], h1 = uc_out[J + 1], h2 = uc_out[J + 2];
    // variable coefficient: faces s-2, s, s+2 (coarse faces J, J+1, J+2 coincide with them)
    double am = 1.0, a0 = 1.0, ap = 1.0;
    if (op_vc(OP)) {
        const double *co = batch_at(a.coef, a.n + 1);
        am = co[s - 2];
        a0 = co[s];
        ap = co[s + 2];
    }
    {
        double Gl = h0 - hm1, Gr = h1 - h0;
        double Fl = f2 - f3, Fr = p0 - f1;
        if (op_vc(OP)) { Gl *= am; Fl *= am; Gr *= a0; Fr *= a0; }
        double tau = (Gl - Gr) - scale2(Fl - Fr, 1);
        if (op_nl(OP)) tau += tau_nl<OP == kOpBratuMx>(scale2(a.lam, -2 * a.M), f2, f1);
        gc_out[J] = scale2(rf[2 * J] + rf[2 * J + 1], rexp) + tau;
    }
    {
        int J2 = J + 1;
        double Gl = h1 - h0, Gr = h2 - h1;
        double Fl = p0 - f1, Fr = p2 - p1;
        if (op_vc(OP)) { Gl *= a0; Fl *= a0; Gr *= ap; Fr *= ap; }
        double tau = (Gl - Gr) - scale2(Fl - Fr, 1);
        if (op_nl(OP)) tau += tau_nl<OP == kOpBratuMx>(scale2(a.lam, -2 * a.M), p0, p1);
        gc_out[J2] = scale2(rf[2 * J2] + rf[2 * J2 + 1], rexp) + tau;
    }
}

// K6: post-smoothing leg of the SR level (Fig. 3, Eq. 5, Fig. 5): full update
// Pi u_{M-1}, then nu2 times (Kaczmarz over the patch's sibling pairs,
// Gauss-Seidel sweep); the segment interior is written out and/or reduced into
// the functionals.  Block x handles segment seg0 + x (seg0 > 0 expands chosen
// segments from the stored coarse solution: PDE decompression on demand).
template <int OP>
__global__ void __launch_bounds__(kSweepBlockMax, 2) sr_post_kernel(SegArgs a) {
    pdl_enter();
    extern __shared__ double sm[];
    const int s = (a.seg0 + blockIdx.x) * a.W;
    const int n = a.n;
    SegSmem m = seg_smem(sm, a, s);
    seg_load(m, a);
    double *p = m.u;
    const double cl = scale2(a.lam, -2 * a.M);
    if (a.uc_corr) {
        // FAS recompute: the pre-smoothed patch as the pre-leg formed it ...
        for (int k = 0; k < a.nu_pre; ++k)
            sweep_op<OP>(p, m.g, cl, m.a, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y);
        // ... with the assembled values in its buffer and frozen cells ...
        const int ne = a.b + 1, seg = a.seg0 + (int)blockIdx.x, nseg = n / a.W;
        const double *ei = batch_at(a.edge_in, (long long)nseg * 2 * ne);
        for (int i = m.lo + (int)threadIdx.x; i < s; i += (int)blockDim.x)
            p[i - m.lo] = ei[(size_t)(seg - 1) * 2 * ne + ne + (i - (s - ne))];
        for (int i = s + a.W + (int)threadIdx.x; i < m.hi; i += (int)blockDim.x)
            p[i - m.lo] = ei[(size_t)(seg + 1) * 2 * ne + (i - (s + a.W))];
        // ... corrected by Eq. 4 with P (u_{M-1} - R ubar) ...
        const int nc = n >> 1;
        double *c2 = sm + a.c2_off;
        stage_coarse_async(m.c, batch_at(a.uc_corr, nc), m.C0, m.C1, nc);
        stage_coarse_async(c2, batch_at(a.uhat, nc), m.C0, m.C1, nc);
        stage_wait();
        __syncthreads();
        fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
        fill_coarse_ghosts(c2, m.C0, m.C1, nc);
        __syncthreads();
        for (int j = m.C0 + (int)threadIdx.x; j < m.C1; j += (int)blockDim.x) m.c[j - m.C0] -= c2[j - m.C0];
        __syncthreads();
        for (int i = m.lo + (int)threadIdx.x; i < m.hi; i += (int)blockDim.x) {
            const int J = i >> 1, nb = (i & 1) ? J + 1 : J - 1;
            p[i - m.lo] += scale2(fma(3.0, m.c[J - m.C0], m.c[nb - m.C0]), -2);
        }
        __syncthreads();
        // ... and smoothed without Kaczmarz
        for (int k = 0; k < a.nu; ++k)
            sweep_op<OP>(p, m.g, cl, m.a, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y);
    } else {
        for (int k = 0; k < a.nu; ++k) {
            // Kaczmarz (Fig. 5): r = u^H_J - (R u)_J added to both children
            for (int J = (m.e0 >> 1) + threadIdx.x; J < (m.e1 >> 1); J += blockDim.x) {
                int i0 = 2 * J - m.lo;
                double r = m.c[J - m.C0] - scale2(p[i0] + p[i0 + 1], -1);
                p[i0] += r;
                p[i0 + 1] += r;
            }
            __syncthreads();
            sweep_op<OP>(p, m.g, cl, m.a, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y);
        }
    }
    const long long s0 = (long long)a.seg0 * a.W;     // first cell of the output
    double *u_out = a.u_out ? batch_at(a.u_out, (long long)gridDim.x * a.W) : nullptr;
    const bool ref = a.fpart && a.u_ref;
    if (ref) {   // the reference of the interior into the rhs array, which the sweeps are done with
        __syncthreads();
        stage_range(m.g + (s - m.lo), batch_at(a.u_ref, a.n) + s, a.W);
        stage_wait();
        __syncthreads();
    }
    FuncAcc q;
    for (int i = s + threadIdx.x; i < s + a.W; i += blockDim.x) {
        const double v = p[i - m.lo];
        if (u_out) u_out[i - s0] = v;
        if (a.fpart) q.add(v, ref ? m.g : nullptr, i - m.lo);
    }
    if (a.fpart) {
        func_block_reduce(q);
        if (threadIdx.x == 0) {
            double *dst = batch_at(a.fpart, (long long)gridDim.x * kNumFunc) + (long long)blockIdx.x * kNumFunc;
#pragma unroll
            for (int k = 0; k < kNumFunc; ++k) dst[k] = q.v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Coarse tail: levels M0..Mc in the shared memory of one block.  Level l
// occupies [2^l - 2^M0, 2^(l+1) - 2^M0) of the u and g arrays.
// mode 0: FMG (Fig. 2) from scratch up to level Mc from g_Mc;
// mode 1: one V-cycle (Fig. 1) on levels Mc..M0 from u_Mc, g_Mc.
// ---------------------------------------------------------------------------
struct TailArgs {
    int M0, Mc, nu1, nu2, mode;
    const double *u_in;        // mode 1: level Mc iterate
    const double *g_in;        // level Mc rhs, scaled by 2^g_exp on load
    int g_exp;
    int *status;               // non-finite f (when g_in is f)
    double *u_out;             // level Mc result
    const double *Ainv;        // inverse of the scaled coarsest operator, row-major
    double lam;                // Bratu: lam (0 otherwise)
    const double *coef[32];    // variable coefficient: face coefficients of level l (2^l + 1 per problem)
};

struct TailSmem {
    double *u, *g, *S, *X, *Y;
    int M0;
    double lam;
    const double *const *coef;  // per-level face coefficients (global), before the batch offset
    __device__ int off(int l) const { return (1 << l) - (1 << M0); }
    // this problem's face coefficients of level l
    __device__ const double *a(int l) const { return coef[l] ? batch_at(coef[l], (1LL << l) + 1) : nullptr; }
};

template <int OP>
__device__ void tail_smooth(TailSmem &m, int l, int nu) {
    const int n = 1 << l;
    double *u = m.u + m.off(l), *g = m.g + m.off(l);
    const double *a = (op_vc(OP)) ? m.a(l) : nullptr;
    for (int k = 0; k < nu; ++k)
        sweep_op<OP, true>(u, g, scale2(m.lam, -2 * l), a, 0, 0, 0, n, n, (k & 1) == 0, m.X, m.Y);
}

// smooth level l, then restriction and tau rhs into level l-1
template <int OP>
__device__ void tail_down(TailSmem &m, int l, int nu) {
    tail_smooth<OP>(m, l, nu);
    const int nc = 1 << (l - 1);
    const double *u = m.u + m.off(l), *g = m.g + m.off(l);
    double *uc = m.u + m.off(l - 1), *gc = m.g + m.off(l - 1);
    for (int J = threadIdx.x; J < nc; J += blockDim.x) {
        int i0 = 2 * J;
        double um2 = (J > 0) ? u[i0 - 2] : 0.0, um1 = (J > 0) ? u[i0 - 1] : 0.0;
        double u2 = (J < nc - 1) ? u[i0 + 2] : 0.0, u3 = (J < nc - 1) ? u[i0 + 3] : 0.0;
        uc[J] = scale2(u[i0] + u[i0 + 1], -1);
        double gcv;
        if (op_vc(OP)) {
            const double *a = m.a(l);
            gcv = tau_rhs_vc(g[i0], g[i0 + 1], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, a[i0], a[i0 + 2]);
        } else {
            gcv = tau_rhs(g[i0], g[i0 + 1], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc);
        }
        if (op_nl(OP)) gcv += tau_nl<OP == kOpBratuMx>(scale2(m.lam, -2 * l), u[i0], u[i0 + 1]);
        gc[J] = gcv;
    }
    __syncthreads();
}

// Coarsest level of the Bratu problem: Newton's method on the scaled system
// T u + c e^u = g (T = h^2 L: tridiag(-1, 2, -1), 3 in the wall rows;
// c = lam h^2) from the current iterate, each step a Thomas solve with the
// Jacobian T + diag(c e^u), until the step is at most 4 ulp of max|u| or stops
// shrinking (at most 100 steps).  One thread; cp and dp hold n scratch values each.
__device__ void coarsest_newton(double *u, const double *g, int n, double c, double *cp, double *dp) {
    double prev = __longlong_as_double(0x7ff0000000000000LL);   // +infinity
    for (int it = 0; it < 100; ++it) {
        // forward elimination of (T + diag(c e^u)) du = g - (T u + c e^u)
        for (int i = 0; i < n; ++i) {
            const double e = c * exp(u[i]);
            const double fl = (i == 0) ? scale2(u[0], 1) : u[i] - u[i - 1];
            const double fr = (i == n - 1) ? -scale2(u[i], 1) : u[i + 1] - u[i];
            const double r = (g[i] - e) - (fl - fr);
            const double diag = ((i == 0 || i == n - 1) ? 3.0 : 2.0) + e;
            const double denom = (i > 0) ? diag + cp[i - 1] : diag;        // lower = -1
            cp[i] = (i < n - 1) ? -1.0 / denom : 0.0;                          // upper = -1
            dp[i] = ((i > 0) ? r + dp[i - 1] : r) / denom;
        }
        double step = 0.0, umax = 0.0, du = dp[n - 1];
        u[n - 1] += du;
        step = fabs(du);
        umax = fabs(u[n - 1]);
        for (int i = n - 2; i >= 0; --i) {
            du = dp[i] - cp[i] * du;
            u[i] += du;
            step = fmax(step, fabs(du));
            umax = fmax(umax, fabs(u[i]));
        }
        if (step <= 4.0 * 2.220446049250313e-16 * umax || step >= prev) break;
        prev = step;
    }
}

template <int OP>
__device__ void tail_coarsest(TailSmem &m, const double *Ainv) {
    if (op_nl(OP)) {
        const int n0 = 1 << m.M0;
        if (threadIdx.x == 0)
            coarsest_newton(m.u + m.off(m.M0), m.g + m.off(m.M0), n0, scale2(m.lam, -2 * m.M0), m.S, m.X);
        __syncthreads();
        return;
    }
    if (op_vc(OP)) {
        const int n0 = 1 << m.M0;
        if (threadIdx.x == 0)
            coarsest_thomas_vc(m.u + m.off(m.M0), m.g + m.off(m.M0), n0, m.a(m.M0), m.S, m.X);
        __syncthreads();
        return;
    }
    const int n0 = 1 << m.M0;
    double *u = m.u + m.off(m.M0);
    const double *g = m.g + m.off(m.M0);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n0; ++j) s = fma(Ainv[i * n0 + j], g[j], s);
        m.S[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) u[i] = m.S[i];
    __syncthreads();
}

// u_l += P (u_{l-1} - R u_l), then smoothing
template <int OP>
__device__ void tail_up(TailSmem &m, int l, int nu) {
    const int n = 1 << l, nc = n >> 1;
    double *u = m.u + m.off(l);
    const double *uc = m.u + m.off(l - 1);
    for (int J = threadIdx.x; J < nc; J += blockDim.x)
        m.S[J] = uc[J] - scale2(u[2 * J] + u[2 * J + 1], -1);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int J = i >> 1, nb = (i & 1) ? J + 1 : J - 1;
        double cn = (nb < 0) ? -m.S[0] : ((nb >= nc) ? -m.S[nc - 1] : m.S[nb]);
        u[i] += scale2(fma(3.0, m.S[J], cn), -2);
    }
    __syncthreads();
    tail_smooth<OP>(m, l, nu);
}

__device__ void tail_interp(TailSmem &m, int l) {
    const int n = 1 << l, nc = n >> 1;
    const double *uc = m.u + m.off(l - 1);
    double *u = m.u + m.off(l);
    // stage the coarse level with two reflected ghosts per side
    for (int j = (int)threadIdx.x - 2; j < nc + 2; j += (int)blockDim.x)
        if (j >= -2) m.S[j + 2] = coarse_reflect(uc, 0, j, nc);
    __syncthreads();
    for (int J = threadIdx.x; J < nc; J += blockDim.x) fmg_interp2(m.S, -2, J, u[2 * J], u[2 * J + 1]);
    __syncthreads();
}

template <int OP>
__global__ void __launch_bounds__(kTailBlock) tail_kernel(const __grid_constant__ TailArgs a) {
    pdl_enter();
    extern __shared__ double sm[];
    TailSmem m;
    m.M0 = a.M0;
    m.lam = a.lam;
    m.coef = a.coef;
    const int tot = (1 << (a.Mc + 1)) - (1 << a.M0);
    m.u = sm;
    m.g = m.u + tot;
    m.S = m.g + tot;
    m.X = m.S + (1 << a.Mc) + 8;
    m.Y = m.X + blockDim.x;
    const int nMc = 1 << a.Mc;
    const double *u_in = batch_at(a.u_in, nMc), *g_in = batch_at(a.g_in, nMc);
    double *u_out = batch_at(a.u_out, nMc);
    stage_range(m.g + m.off(a.Mc), g_in, nMc);
    if (a.mode == 1) stage_range(m.u + m.off(a.Mc), u_in, nMc);
    stage_wait();
    __syncthreads();
    bool bad = false;
    if (a.g_exp)
        for (int i = threadIdx.x; i < nMc; i += blockDim.x) {
            bad = bad || nonfinite(m.g[m.off(a.Mc) + i]);
            m.g[m.off(a.Mc) + i] = scale2(m.g[m.off(a.Mc) + i], a.g_exp);
        }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && a.status) atomicOr(a.status, kStatusNonFinite);
    if (a.mode == 0) {
        for (int l = a.Mc; l > a.M0; --l) {
            const double *g = m.g + m.off(l);
            double *gc = m.g + m.off(l - 1);
            for (int J = threadIdx.x; J < (1 << (l - 1)); J += blockDim.x)
                gc[J] = scale2(g[2 * J] + g[2 * J + 1], 1);
            __syncthreads();
        }
        // the first coarsest solve of the FMG starts from zero (Newton needs a
        // starting iterate; the linear solve ignores it)
        for (int i = threadIdx.x; i < (1 << a.M0); i += blockDim.x) m.u[m.off(a.M0) + i] = 0.0;
        __syncthreads();
        tail_coarsest<OP>(m, a.Ainv);
        for (int k = a.M0; k < a.Mc; ++k) {
            tail_interp(m, k + 1);
            for (int l = k + 1; l > a.M0; --l) tail_down<OP>(m, l, a.nu1);
            tail_coarsest<OP>(m, a.Ainv);
            for (int l = a.M0 + 1; l <= k + 1; ++l) tail_up<OP>(m, l, a.nu2);
        }
    } else {
        for (int l = a.Mc; l > a.M0; --l) tail_down<OP>(m, l, a.nu1);
        tail_coarsest<OP>(m, a.Ainv);
        for (int l = a.M0 + 1; l <= a.Mc; ++l) tail_up<OP>(m, l, a.nu2);
    }
    for (int i = threadIdx.x; i < nMc; i += blockDim.x) u_out[i] = m.u[m.off(a.Mc) + i];
}

}  // namespace srfmg
