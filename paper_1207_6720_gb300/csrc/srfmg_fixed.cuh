// srfmg_fixed.cuh -- sm_103a kernels of the FMG-FAS-SR solve in 64-bit fixed
// point (the SRFMG_MIXED precision).
//
// GB300 executes FP64 at about 1/70 of its FP32 rate, while 64-bit integer
// adds run about 30 times faster than FP64 adds and 64-bit shifts and small
// multiplies about 10 times faster (measured).  Here the quantities whose
// accuracy the method depends on -- the solution, the residual, the tau
// correction and the FMG interpolation -- are 64-bit fixed-point integers:
//   u  = U * 2^-S                 on every level,
//   g_l = G * 2^-(Sg0 + 2l)       (scaled right-hand side h_l^2 rhs_l),
// with S = 62 - E and Sg0 = 60 - E, where 2^E bounds max|f| (computed on the
// device before the solve).  |u| <= max|f|/8 keeps |U| below 2^59 with eight
// times headroom, and |G| below 2^60; relative to the largest value every
// quantity carries at least 59 bits (FP64: 53).  Sums and differences are
// exact; the tau correction (differences of differences of u) is exact; the
// only roundings are the explicit halvings of the smoother, the restriction,
// the prolongations and the FMG interpolation (half a unit each, far below the
// FP64 rounding of the same quantities).  Corrections stay integers too:
// converting between integers and floating point costs as much as an FP64
// operation on this part.  The coarsest-level direct solve stays in FP64.
// f (input) and u (output) are FP64; they are converted with integer bit
// operations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace srfmg {
namespace fx {

typedef long long i64;
typedef unsigned long long u64;

// Fixed-point scales of one solve, written on the device by scale_kernel
// (S, Sg0, E) and, for the variable coefficient, by coef_scale_kernel (Ka, Ea,
// Kb).
struct Scale {
    int S;       // u = U 2^-S
    int Sg0;     // g_l = G 2^-(Sg0 + 2l)
    int E;       // max|f| < 2^E
    int Ka;      // variable coefficient: 2^Ka >= 1 / min a', a' = a 2^-Ea (0 otherwise)
    // scale_kernel's accumulators: zero between solves (set at plan creation,
    // restored by the kernel's last block)
    int emax;           // largest biased exponent field of f seen so far
    unsigned done;      // blocks of this problem that have finished
    int Ea;      // variable coefficient: max a < 2^Ea
    int Kb;      // variable coefficient: 62 - Ka, the scale of the reciprocal diagonals
};

// x / 2^k rounded half up, 0 < k < 63.
__device__ __forceinline__ i64 shr_round(i64 x, int k) { return (x + (1LL << (k - 1))) >> k; }

// round(x 2^k) for a double x with |x 2^k| < 2^62 (subnormals read as 0).
__device__ __forceinline__ i64 f64_to_fixed(double x, int k) {
    u64 b = (u64)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;
    i64 m = (i64)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));   // |x| = m 2^(e-1075)
    int sh = e - 1075 + k;
    i64 v;
    if (sh >= 0) v = m << sh;
    else if (sh > -63) v = (m + (1LL << (-sh - 1))) >> (-sh);
    else v = 0;
    return (b >> 63) ? -v : v;
}

// U 2^-S as the nearest double (ties to even), for |U| < 2^59.  m = |U| has
// its leading one at bit p; above 53 significant bits it is rounded by adding
// half a unit minus one plus the lowest kept bit and truncating (ties go to the
// even quotient), and the 53-bit q (implicit one at bit 52, or 2^53 after a
// rounding carry) is added to the exponent field (p - S + 1022) << 52, so that
// a carry out of the mantissa raises the exponent by itself.
__device__ __forceinline__ double fixed_to_f64(i64 U, int S) {
    const u64 sign = (u64)U & (1ULL << 63);
    const u64 m = sign ? (u64)0 - (u64)U : (u64)U;
    const int p = 63 - __clzll((long long)(m | 1));
    u64 q;
    if (p > 52) {
        const int sh = p - 52;
        q = (m + ((1ULL << (sh - 1)) - 1) + ((m >> sh) & 1)) >> sh;
    } else {
        q = m << (52 - p);
    }
    const u64 b = sign | ((((u64)(p - S + 1022)) << 52) + q);
    return __longlong_as_double((long long)(U == 0 ? 0ULL : b));
}

// Fourth order FMG interpolation Pi (Sec. 4) in fixed point: 128 Pi is the
// integer combination (-5, 35, 105, -7) (or its mirror) of coarse cells
// J-2..J+1 (J-1..J+2), rounded to the nearest unit.  Both children of coarse
// cell J are formed together, without 128-bit products: with U = 16a + b
// (0 <= b < 16), sum w U = 16 Sa + Sb where Sa = sum w a fits 64 bits for
// |U| < 2^59 (sum |w| = 152 < 2^8) and |Sb| <= 152 * 15; then
//   floor((16 Sa + Sb + 64) / 128) = (Sa + ((Sb + 64) >> 4)) >> 3
// exactly (the dropped remainder of (Sb + 64) / 16 is below 1/8 of the last
// shift's unit).  c[j - cbase] holds coarse cells J-2..J+2.
__device__ __forceinline__ void fmg_interp2(const i64 *c, int cbase, int J, i64 &left, i64 &right) {
    const i64 *p = c + (J - cbase);
    i64 a[5];
    int b[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const i64 v = p[j - 2];
        a[j] = v >> 4;
        b[j] = (int)(v & 15);
    }
    const i64 sal = -5 * a[0] + 35 * a[1] + 105 * a[2] - 7 * a[3];
    const i64 sar = -7 * a[1] + 105 * a[2] + 35 * a[3] - 5 * a[4];
    const int sbl = -5 * b[0] + 35 * b[1] + 105 * b[2] - 7 * b[3] + 64;
    const int sbr = -7 * b[1] + 105 * b[2] + 35 * b[3] - 5 * b[4] + 64;
    left = (sal + (i64)(sbl >> 4)) >> 3;
    right = (sar + (i64)(sbr >> 4)) >> 3;
}

// x / 3 rounded toward zero (C division) for |x| < 2^63: the high word of
// x (2^64 + 2) / 3, plus one for negative x.
__device__ __forceinline__ i64 div3(i64 x) {
    return __mul64hi(x, 0x5555555555555556LL) + (x < 0 ? 1 : 0);
}

// Lexicographic Gauss-Seidel sweep in place, fixed point; the structure of the
// FP64 lex_sweep (srfmg_kernels.cuh): residual r_i = gs_i - (F_{i-1/2} -
// F_{i+1/2}) with the right-hand side already in solution units (gs),
// correction recurrence delta_i = (r_i + delta_{i-1}) / 2 rounded half up
// (wall cells / 3), update U += delta.  Chunks of C cells, one per thread
// (the number of chunks of [lo, hi) must not exceed blockDim.x); the carry
// into a chunk is the fixed sum over the chunks that reach 64 cells back: a
// shift by 64 or more leaves nothing of a 63-bit value, so dropping those
// terms changes nothing.  Integer sums are exact, so the residual is written
// gs + u_{q-1} + u_{q+1} - 2 u_q in either direction.  SHIFT: gs holds the
// level's G and each value is moved into solution units on load,
// shr_round(G, gsh) (the same values as a pre-shifted array, without the pass
// that would form it).
template <int C, bool PRELOAD, bool ASC, bool SHIFT = false>
__device__ __noinline__ void lex_sweep_dir(i64 *__restrict__ u, const i64 *__restrict__ gs, int base, int lo,
                                              int hi, int n, i64 *X, int gsh = 0) {
    auto G = [gsh](i64 x) { return SHIFT ? shr_round(x, gsh) : x; };
    constexpr int s = ASC ? 1 : -1;                // sweep position q is u[a0 + s q]
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
    // a warp whose chunks are all full and away from the walls takes the
    // straight-line path (no clamps, no range selects)
    const bool fast = __all_sync(0xffffffffu, !active || (k0 == 0 && k1 == C && !wall0 && !wall1));
    i64 rr[C];
    i64 p = 0, r_end = 0;
    if (active) {
        i64 w[C + 2];
        if (fast) {
            const i64 *up = u + (a0 + s * (q0 - 1)), *gp = gs + (a0 + s * q0);
#pragma unroll
            for (int j = 0; j < C + 2; ++j) w[j] = up[s * j];
#pragma unroll
            for (int k = 0; k < C; ++k) {
                p = (G(gp[s * k]) + w[k] + w[k + 2] - 2 * w[k + 1] + p + 1) >> 1;
                rr[k] = p;
            }
        } else {
#pragma unroll
            for (int j = 0; j < C + 2; ++j) w[j] = u[a0 + s * min(max(q0 - 1 + j, qmin), qmax)];
            if (wall0) p = div3(G(gs[a0]) + w[2] - 3 * w[1]);
            if (wall1) r_end = G(gs[a0 + s * (n - 1)]) + u[a0 + s * (n - 2)] - 3 * u[a0 + s * (n - 1)];
            i64 gv[C];
#pragma unroll
            for (int k = 0; k < C; ++k) gv[k] = G(gs[a0 + s * min(max(q0 + k, qmin), qmax)]);
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const i64 r = gv[k] + w[k] + w[k + 2] - 2 * w[k + 1];
                const i64 pn = (r + p + 1) >> 1;
                p = (k >= ka && k < kb) ? pn : p;
                rr[k] = p;
            }
        }
        X[t] = p;
    }
    __syncthreads();
    if (active) {
        constexpr int J = (64 + C - 1) / C - 1;
        i64 cin = 0;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const int idx = t - 1 - j;
            const i64 x = X[max(idx, 0)];
            cin = (cin >> C) + (idx >= 0 ? x : 0);
        }
        // PRELOAD: all loads first, then the arithmetic, then the stores (a
        // load after a store to a runtime-indexed address waits for the
        // store), for latency-bound blocks; otherwise the increments are
        // added in place, which needs fewer registers.
        if (fast) {
            i64 *up = u + (a0 + s * q0);
            i64 uo[C];
#pragma unroll
            for (int k = 0; k < C; ++k) uo[k] = PRELOAD ? up[s * k] : 0;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                if (PRELOAD) up[s * k] = uo[k] + rr[k] + (cin >> (k + 1));
                else up[s * k] += rr[k] + (cin >> (k + 1));
            }
        } else {
            i64 uo[C];
#pragma unroll
            for (int k = 0; k < C; ++k) uo[k] = PRELOAD ? u[a0 + s * min(max(q0 + k, qmin), qmax)] : 0;
            const i64 ue = u[wall1 ? a0 + s * (n - 1) : a0 + s * min(max(q0, qmin), qmax)];   // in range
            i64 c = cin, dl = cin;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                if (k >= k0) c >>= 1;                 // cin >> (k-k0+1)
                dl = (k >= k0 && k < kb) ? rr[k] + c : dl;
                uo[k] += dl;
            }
#pragma unroll
            for (int k = 0; k < C; ++k)
                if (k >= k0 && k < kb) {
                    if (PRELOAD) u[a0 + s * (q0 + k)] = uo[k];
                    else u[a0 + s * (q0 + k)] += uo[k];
                }
            if (wall1) u[a0 + s * (n - 1)] = ue + div3(r_end + dl);
        }
    }
    __syncthreads();
}

template <int C, bool PRELOAD = false, bool SHIFT = false>
__device__ __forceinline__ void lex_sweep(i64 *__restrict__ u, const i64 *__restrict__ gs, int base, int lo,
                                          int hi, int n, bool asc, i64 *X, int gsh = 0) {
    if (asc) lex_sweep_dir<C, PRELOAD, true, SHIFT>(u, gs, base, lo, hi, n, X, gsh);
    else lex_sweep_dir<C, PRELOAD, false, SHIFT>(u, gs, base, lo, hi, n, X, gsh);
}

// tau-corrected coarse right-hand side (Eqs. 6-7), exact: the tau term is a
// combination of differences of u in solution units, moved into the coarse
// right-hand side's units by a left shift of tsh = 2l - 4 bits and added to
// gr, the restricted right-hand side (the mean of the two children in the
// coarse units, rounded half up: restrict_rhs).  um2..u3: U at fine cells
// 2J-2 .. 2J+3.  tau is moved by a multiplication with 2^tsh (a shift that is
// defined for negatives).
__device__ __forceinline__ i64 restrict_rhs(i64 g0, i64 g1) { return (g0 + g1 + 1) >> 1; }
__device__ __forceinline__ i64 tau_rhs(i64 gr, i64 um2, i64 um1, i64 u0, i64 u1, i64 u2, i64 u3,
                                       int J, int nc, int tsh) {
    i64 hJ = (u0 + u1) >> 1;
    i64 Gl = (J == 0) ? 2 * hJ : hJ - ((um2 + um1) >> 1);
    i64 Gr = (J == nc - 1) ? -2 * hJ : ((u2 + u3) >> 1) - hJ;
    i64 Fl = (J == 0) ? 2 * u0 : u0 - um1;
    i64 Fr = (J == nc - 1) ? -2 * u1 : u2 - u1;
    i64 tau = (Gl - Gr) - 2 * (Fl - Fr);
    return gr + tau * (1LL << tsh);
}

// tau_rhs of a coarse cell away from both walls, without the wall cases, the
// same integers: (Gl - Gr) = 2 hJ - h_{J-1} - h_{J+1} and (Fl - Fr) = (u0 + u1)
// - (um1 + u2).
__device__ __forceinline__ i64 tau_rhs_interior(i64 gr, i64 um2, i64 um1, i64 u0, i64 u1, i64 u2, i64 u3, int tsh) {
    const i64 hm = (um2 + um1) >> 1, h = (u0 + u1) >> 1, hp = (u2 + u3) >> 1;
    const i64 tau = (2 * h - hm - hp) - 2 * ((u0 + u1) - (um1 + u2));
    return gr + tau * (1LL << tsh);
}

// --------------------------------------------------------------------------
// Variable coefficient -(a u')' = f in fixed point.
//
// The operator is normalised by an exact power of two, a' = a 2^-Ea with
// max a < 2^Ea, and the right-hand side with it (G carries 2^-Ea, folded into
// Sg0), which leaves u unchanged; 1/2 <= max a' < 1 and min a' >= 2^-Ka.
// Per level, the face coefficients are A = round(a' 2^61) (at least 52 bits
// for a contrast max a / min a below 2^8), and each cell keeps its Gauss-Seidel
// multipliers in two words: the reciprocal diagonal b = 1/(a'_near + a'_far) as
// round(b 2^(62 - Ka)) and the ascending multiplier m = a'_left / (a'_left +
// a'_right) as round(m 2^63) (a wall face counts twice; the descending
// multiplier is 2^63 - m).  The fluxes a' (U_{i+1} - U_i) are exact 128-bit
// products rounded to units (half a unit each, as the rounding of the
// right-hand side into solution units), and tau keeps the coarse right-hand
// side's finer grid; every product that enters a correction is an exact
// 128-bit product rounded to the nearest unit (a biased rounding of a few units
// per cell would act as a smooth right-hand side on the fine levels, whose
// right-hand side in solution units is small, and reach the coarse levels
// through tau at the walls).  The scale S = 61 - E + Ea - Ka bounds |U| below
// 2^59: with the Green's function of -(a'u')' = f', |u| <= max|f'| / (4 min a').
// --------------------------------------------------------------------------
constexpr int kSaVc = 61;           // A = round(a' 2^61)
constexpr int kKaMax = 9;           // contrast max a / min a below 2^8


// round(A d / 2^sh) (half away from zero) for A < 2^62, 1 <= sh <= 63, an exact
// 128-bit product; |result| < 2^63
__device__ __forceinline__ i64 mul_shr_round(u64 A, i64 d, int sh) {
    const u64 ad = d < 0 ? (u64)0 - (u64)d : (u64)d;
    const u64 lo = A * ad;
    u64 hi = __umul64hi(A, ad);
    const u64 lo2 = lo + (1ULL << (sh - 1));
    hi += (lo2 < lo) ? 1ULL : 0ULL;
    const u64 r = (hi << (64 - sh)) | (lo2 >> sh);
    return d < 0 ? -(i64)r : (i64)r;
}

// Signed 128-bit product A d (two's complement hi:lo)
struct S128 {
    u64 lo;
    u64 hi;
};
__device__ __forceinline__ S128 mul_s128(u64 A, i64 d) {
    const u64 ad = d < 0 ? (u64)0 - (u64)d : (u64)d;
    S128 r;
    r.lo = A * ad;
    r.hi = __umul64hi(A, ad);
    if (d < 0) {
        r.lo = ~r.lo + 1ULL;
        r.hi = ~r.hi + (r.lo == 0 ? 1ULL : 0ULL);
    }
    return r;
}
// round((a - b) / 2^k) for 1 <= k <= 63 when the result fits 64 bits
__device__ __forceinline__ i64 s128_diff_shr_round(S128 a, S128 b, int k) {
    const u64 lo = a.lo - b.lo;
    u64 hi = a.hi - b.hi - (a.lo < b.lo ? 1ULL : 0ULL);
    const u64 lo2 = lo + (1ULL << (k - 1));
    hi += (lo2 < lo) ? 1ULL : 0ULL;
    return (i64)((hi << (64 - k)) | (lo2 >> k));
}

// Lexicographic Gauss-Seidel sweep of -(a u')' = f in place, fixed point, with
// the layout and chunking of lex_sweep_dir: the residual of the old values
//   r_q = gs_q - (F_near - F_far),  F = round(A (U_{q} - U_{q-1}) / 2^61)
// (sweep coordinates; the odd ghost -U at both walls), the correction
// recurrence delta_q = b_q r_q + m_q delta_{q-1}, an affine recurrence whose
// chunk carries are the nested sum over the 11 preceding chunks
// (X_{c-1} + Y_{c-1}(X_{c-2} + ...), Y the product of a chunk's multipliers, as
// in the FP64 variable-coefficient sweep: multipliers <= 0.6 over 99 cells
// leave less than one unit of a 64-bit value), update U += delta.
// A[f - abase]: faces of the staged range; BM[i - base]: the cells'
// multipliers (two words per cell).  X, Y: one word per thread each.  SHIFT as
// in lex_sweep_dir.
constexpr int kTruncVcFx = 96;

template <int C, bool ASC, bool SHIFT = false>
__device__ __noinline__ void lex_sweep_vc_dir(i64 *__restrict__ u, const i64 *__restrict__ gs,
                                              const u64 *__restrict__ A, const u64 *__restrict__ BM, int base,
                                              int abase, int lo, int hi, int n, i64 *X, i64 *Y, int Kb,
                                              int gsh = 0) {
    auto G = [gsh](i64 x) { return SHIFT ? shr_round(x, gsh) : x; };
    constexpr int s = ASC ? 1 : -1;
    const int t = threadIdx.x;
    const int qlo = ASC ? lo : n - hi, qhi = ASC ? hi : n - lo;
    const int c_first = qlo / C, nch = (qhi - 1) / C - c_first + 1;
    const bool active = t < nch;
    const int q0 = (c_first + t) * C;
    const int k0 = max(qlo - q0, 0), k1 = min(qhi - q0, C);
    const int qmin = max(qlo - 1, 0), qmax = min(qhi, n - 1);
    const int a0 = ASC ? -base : n - 1 - base;      // cell of position q: a0 + s q
    const int f0 = ASC ? -abase : n - abase;        // face before position q: f0 + s q
    i64 rr[C];
    u64 aa[C];
    i64 p = 0;
    u64 yp = 1ULL << 62;                           // the chunk's product of multipliers, scaled by 2^62
    if (active) {
        i64 wp = u[a0 + s * min(max(q0 - 1, qmin), qmax)];
        if (q0 == 0 && qlo == 0) wp = -u[a0];                            // odd ghost at the first wall
        i64 wc = u[a0 + s * min(max(q0, qmin), qmax)];
        i64 Fn = mul_shr_round(A[f0 + s * min(max(q0, qlo), qhi)], wc - wp, kSaVc);
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const int q = q0 + k;
            i64 wn = u[a0 + s * min(max(q + 1, qmin), qmax)];
            if (q + 1 >= n) wn = -wc;                                    // odd ghost at the last wall
            const i64 Ff = mul_shr_round(A[f0 + s * min(max(q + 1, qlo), qhi)], wn - wc, kSaVc);
            const i64 r = G(gs[a0 + s * min(max(q, qmin), qmax)]) - (Fn - Ff);
            const int ci = 2 * (a0 + s * min(max(q, qmin), qmax));
            const u64 B = BM[ci], ma = BM[ci + 1];
            const u64 m = ASC ? ma : (1ULL << 63) - ma;
            const bool in = k >= k0 && k < k1;
            p = in ? mul_shr_round(B, r, Kb) + mul_shr_round(m, p, 63) : p;
            yp = in ? __umul64hi(yp, m) << 1 : yp;   // relative error 2^-62: the carries' weights
            rr[k] = p;
            aa[k] = yp;
            Fn = Ff;
            wc = wn;
        }
        X[t] = p;
        Y[t] = (i64)yp;
    }
    __syncthreads();
    if (active) {
        constexpr int J = (kTruncVcFx + C - 1) / C - 1;
        i64 cin = 0;
#pragma unroll
        for (int j = J; j >= 0; --j) {
            const int idx = t - 1 - j;
            const i64 x = X[max(idx, 0)];
            const u64 y = (u64)Y[max(idx, 0)];
            cin = idx >= 0 ? x + mul_shr_round(y, cin, 62) : 0;
        }
        i64 uo[C];
#pragma unroll
        for (int k = 0; k < C; ++k) uo[k] = u[a0 + s * min(max(q0 + k, qmin), qmax)];
#pragma unroll
        for (int k = 0; k < C; ++k)
            if (k >= k0 && k < k1) u[a0 + s * (q0 + k)] = uo[k] + rr[k] + mul_shr_round(aa[k], cin, 62);
    }
    __syncthreads();
}

template <int C, bool SHIFT = false>
__device__ __forceinline__ void lex_sweep_vc(i64 *__restrict__ u, const i64 *__restrict__ gs, const u64 *A,
                                             const u64 *BM, int base, int abase, int lo, int hi, int n, bool asc,
                                             i64 *X, i64 *Y, int Kb, int gsh = 0) {
    if (asc) lex_sweep_vc_dir<C, true, SHIFT>(u, gs, A, BM, base, abase, lo, hi, n, X, Y, Kb, gsh);
    else lex_sweep_vc_dir<C, false, SHIFT>(u, gs, A, BM, base, abase, lo, hi, n, X, Y, Kb, gsh);
}

// tau-corrected coarse right-hand side of -(a u')' = f (Eqs. 6-7 with the
// level's own coefficients): the terms of tau_rhs weighted by the fine faces
// 2J (left) and 2J + 2 (right), which the coarse faces J and J + 1 coincide
// with, as one exact 128-bit combination moved into the coarse right-hand
// side's units (2^tsh solution units) and rounded there.
__device__ __forceinline__ i64 tau_rhs_vc(i64 gr, i64 um2, i64 um1, i64 u0, i64 u1, i64 u2, i64 u3, int J, int nc,
                                          int tsh, u64 AL, u64 AR) {
    const i64 hJ = (u0 + u1) >> 1;
    const i64 Gl = (J == 0) ? 2 * hJ : hJ - ((um2 + um1) >> 1);
    const i64 Gr = (J == nc - 1) ? -2 * hJ : ((u2 + u3) >> 1) - hJ;
    const i64 Fl = (J == 0) ? 2 * u0 : u0 - um1;
    const i64 Fr = (J == nc - 1) ? -2 * u1 : u2 - u1;
    return gr + s128_diff_shr_round(mul_s128(AL, Gl - 2 * Fl), mul_s128(AR, Gr - 2 * Fr), kSaVc - tsh);
}

// The fixed-point coefficient of every level from the FP64 face coefficients
// (coef_hierarchy_kernel's output): coef_scale_kernel (one block per problem)
// reduces max a and min a over the finest level's faces into Ea, Ka, Kb and
// flags a contrast beyond 2^8; coef_fixed_kernel (grid-stride over the faces
// of every level, problem blockIdx.y) writes A and the packed multipliers.
struct CoefFxArgs {
    const double *coef[32];    // FP64 a per level (2^l + 1 faces per problem)
    u64 *A[32];                // round(a 2^(61 - Ea)) per face
    u64 *BM[32];               // multipliers per cell, two words each
    Scale *sc;
    int *bad;
    int M, M0;
};

__global__ void coef_scale_kernel(CoefFxArgs a) {
    const long long nf = (1LL << a.M) + 1;
    const double *c = a.coef[a.M] + (long long)blockIdx.x * nf;
    // a > 0: the bit patterns of positive doubles order like the values
    long long mx = 0, mn = 0x7fefffffffffffffLL;
    for (long long j = threadIdx.x; j < nf; j += blockDim.x) {
        const long long b = __double_as_longlong(c[j]);
        mx = b > mx ? b : mx;
        mn = b < mn ? b : mn;
    }
    __shared__ long long smx[32], smn[32];
    for (int o = 16; o > 0; o >>= 1) {
        const long long x = __shfl_xor_sync(0xffffffffu, mx, o), y = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = x > mx ? x : mx;
        mn = y < mn ? y : mn;
    }
    if ((threadIdx.x & 31) == 0) {
        smx[threadIdx.x >> 5] = mx;
        smn[threadIdx.x >> 5] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mx = smx[w] > mx ? smx[w] : mx;
            mn = smn[w] < mn ? smn[w] : mn;
        }
        // 2^(e-1) <= x < 2^e with e = biased exponent - 1022
        const int Ea = (int)((mx >> 52) & 0x7ff) - 1022;
        const int emin = (int)((mn >> 52) & 0x7ff) - 1022;
        int Ka = Ea - emin + 1;                    // 1 / min a' <= 2^(Ea - emin + 1)
        // contrast below 2^8 keeps Ka <= 9 (A with at least 52 bits)
        if (!(__longlong_as_double(mx) < 256.0 * __longlong_as_double(mn)) || Ka > kKaMax) {
            atomicOr(a.bad, 1);
            Ka = kKaMax;
        }
        Scale *sc = a.sc + blockIdx.x;
        sc->Ea = Ea;
        sc->Ka = Ka;
        sc->Kb = 62 - Ka;
    }
}

__global__ void coef_fixed_kernel(CoefFxArgs a) {
    const Scale *sc = a.sc + blockIdx.y;
    const int Ea = sc->Ea, Ka = sc->Ka;
    for (int l = a.M; l >= a.M0; --l) {
        const long long n = 1LL << l;
        const double *c = batch_at(a.coef[l], n + 1);
        u64 *A = batch_at(a.A[l], n + 1), *BM = batch_at(a.BM[l], 2 * n);
        for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j <= n;
             j += (long long)gridDim.x * blockDim.x) {
            A[j] = (u64)f64_to_fixed(c[j], kSaVc - Ea);
            if (j < n) {
                const double al = (j == 0) ? 2.0 * c[0] : c[j];
                const double ar = (j == n - 1) ? 2.0 * c[n] : c[j + 1];
                const double D = al + ar;
                BM[2 * j] = (u64)rint(scale2(1.0 / D, Ea + 62 - Ka));   // b' 2^(62 - Ka) < 2^61
                BM[2 * j + 1] = (u64)rint(scale2(al / D, 63));          // m 2^63, m <= 256/257
            }
        }
    }
}

// --------------------------------------------------------------------------
// Scale: E with max|f| < 2^E from the largest exponent field of f.
// --------------------------------------------------------------------------
// (one Scale per problem of a batch: sc[blockIdx.y])
// One launch: every block reduces the exponent fields of its part of f (16-byte
// loads; n is even and f 16-byte aligned) into sc->emax; the last block of the
// problem to finish (a counter, after a fence) turns the maximum into E, S and
// Sg0 and restores the accumulators to zero for the next solve.  An inf or
// NaN in f (exponent field 0x7ff) is recorded in the status word.
__global__ void scale_kernel(const double *f, long long n, Scale *sc, int *status, int vc) {
    pdl_enter();
    const double2 *f2 = reinterpret_cast<const double2 *>(batch_at(f, n));
    sc += blockIdx.y;
    int emax = 0;
    const long long n2 = n >> 1, stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i + 7 * stride < n2; i += 8 * stride) {     // eight 16-byte loads in flight per thread
        double2 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = f2[i + k * stride];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            emax = max(emax, (int)((__double_as_longlong(v[k].x) >> 52) & 0x7ff));
            emax = max(emax, (int)((__double_as_longlong(v[k].y) >> 52) & 0x7ff));
        }
    }
    for (; i < n2; i += stride) {
        const double2 v = f2[i];
        emax = max(emax, (int)((__double_as_longlong(v.x) >> 52) & 0x7ff));
        emax = max(emax, (int)((__double_as_longlong(v.y) >> 52) & 0x7ff));
    }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&sc->emax, emax);
        if (emax == 0x7ff && status) atomicOr(status, kStatusNonFinite);   // inf or NaN in f
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&sc->done, 1u) == gridDim.x - 1) {
        __threadfence();
        const int raw = atomicExch(&sc->emax, 0);
        sc->done = 0;
        int E = raw - 1022;                      // 2^E bounds max|f| (raw 0: f = 0)
        E = E < -100 ? -100 : (E > 900 ? 900 : E);
        sc->E = E;
        if (vc) {                                // -(a u')' = f: |u| <= max|f'| / (4 min a'), f' = f 2^-Ea
            sc->S = 61 - E + sc->Ea - sc->Ka;
            sc->Sg0 = sc->S - 2 - sc->Ea;
        } else {
            sc->S = 62 - E;
            sc->Sg0 = 60 - E;
        }
    }
}

// --------------------------------------------------------------------------
// Right-hand side hierarchy: G on levels lin-1 .. lstop; level lin is f
// (converted) when from_f, else the fixed-point array `in`.
// --------------------------------------------------------------------------
struct RhsArgs {
    const double *f;
    const i64 *in;
    const Scale *sc;
    int from_f, lin, lstop, depth;
    int chunk_log;             // log2 of the cells each block reduces (>= depth)
    i64 *out[32];
};

__global__ void rhs_hierarchy_kernel(RhsArgs a) {
    pdl_enter();
    extern __shared__ i64 smi[];
    const int chunk = 1 << a.chunk_log;       // cells of level lin per block (>= 2^depth)
    i64 *cur = smi, *nxt = smi + chunk;
    const long long base = (long long)blockIdx.x * chunk;
    const Scale *sc = a.sc + blockIdx.y;
    const double *f = batch_at(a.f, 1LL << a.lin);
    const i64 *in = batch_at(a.in, 1LL << a.lin);
    const int k = sc->Sg0;                // f 2^-2M 2^(Sg0+2M) = f 2^Sg0
    if (a.from_f) stage_range(cur, f + base, chunk);
    else stage_range(cur, in + base, chunk);
    stage_wait();
    __syncthreads();
    if (a.from_f)
        for (int i = threadIdx.x; i < chunk; i += blockDim.x) cur[i] = f64_to_fixed(__longlong_as_double(cur[i]), k);
    __syncthreads();
    int len = chunk;
    for (int l = a.lin; l > a.lstop && len > 1; --l) {
        const int half = len >> 1;
        i64 *dst = batch_at(a.out[l - 1], 1LL << (l - 1)) + (base >> (a.lin - l + 1));
        for (int J = threadIdx.x; J < half; J += blockDim.x) {
            i64 x = (cur[2 * J] + cur[2 * J + 1] + 1) >> 1;
            nxt[J] = x;
            dst[J] = x;
        }
        __syncthreads();
        i64 *tmp = cur; cur = nxt; nxt = tmp;
        len = half;
    }
}

// --------------------------------------------------------------------------
// Stored-level passes (tile + halo, global lexicographic smoothing).
// --------------------------------------------------------------------------
struct LevelArgs {
    int l, n, tile, halo, nu;
    int maxlen, maxc, maxch;
    const Scale *sc;
    const i64 *u_src;          // level l iterate, or level l-1 for the FMG interpolation
    const i64 *g;              // G_l; NULL on the finest level (read f instead)
    const double *f;
    const i64 *uc_src;         // up pass: corrected level l-1
    i64 *u_out;                // level l after the pass (tile), when u_out_f64 is NULL
    double *u_out_f64;         // finest level without SR: the FP64 solution
    i64 *uc_out, *gc_out;      // down pass: restricted solution and tau rhs on level l-1
    const u64 *cA, *cBM;       // variable coefficient: this level's A (faces) and multipliers (cells)
    const double *u_src_f64;   // down pass of a further V-cycle on the finest level of a plan
                               // without SR: the caller's FP64 solution (instead of u_src)
};

// Shared memory: u, gs (staged G or f, then the right-hand side in solution
// units), the coarse cells, the chunk carries, gr (restricted G of the tile's
// coarse cells, down pass): 2 maxlen + 2 maxc + maxch words; the variable
// coefficient adds A (maxlen + 1 faces), BM (two words per cell) and the
// carries' Y (maxch): 3 maxlen + 1 + maxch words more.
struct LevelSmem {
    i64 *u, *gs, *c, *X, *gr, *Y;
    u64 *A, *BM;
    int gsh;                   // > 0: gs holds G_l, shifted into solution units by the sweeps
    int L0, L1, C0, C1;
    // this problem's arrays (see batch_at)
    const Scale *sc;
    const i64 *usrc, *gin, *ucsrc;
    const double *fin;
    i64 *uout, *ucout, *gcout;
    double *uout64;
};

// Layout and this problem's arrays (see batch_at); u_src is on level l-1
// when it feeds the FMG interpolation.
__device__ __forceinline__ LevelSmem level_smem(i64 *sm, int s, const LevelArgs &a, bool u_src_coarse) {
    LevelSmem m;
    m.L0 = max(0, s - a.halo);
    m.L1 = min(a.n, s + a.tile + a.halo);
    m.C0 = (m.L0 >> 1) - 2;
    m.C1 = ((m.L1 - 1) >> 1) + 3;
    m.u = sm;
    m.gs = m.u + a.maxlen;
    m.c = m.gs + a.maxlen;
    m.X = m.c + a.maxc;
    m.gr = m.X + a.maxch;
    m.A = (u64 *)(m.gr + a.maxc);
    m.BM = m.A + a.maxlen + 1;
    m.Y = (i64 *)(m.BM + 2 * a.maxlen);
    const long long n = a.n;
    m.sc = a.sc + blockIdx.y;
    m.usrc = batch_at(a.u_src, u_src_coarse ? n / 2 : n);
    m.gin = batch_at(a.g, n);
    m.fin = batch_at(a.f, n);
    m.ucsrc = batch_at(a.uc_src, n / 2);
    m.uout = batch_at(a.u_out, n);
    m.uout64 = batch_at(a.u_out_f64, n);
    m.ucout = batch_at(a.uc_out, n / 2);
    m.gcout = batch_at(a.gc_out, n / 2);
    return m;
}

// Issue the staging copies of G_l (or of f, converted by prepare_rhs) and,
// for the variable coefficient, of the level's A and multipliers.
template <bool VC>
__device__ void stage_g_async(LevelSmem &m, const LevelArgs &a) {
    if (m.gin) stage_range(m.gs, m.gin + m.L0, m.L1 - m.L0);
    else stage_range(m.gs, m.fin + m.L0, m.L1 - m.L0);
    if (VC) {
        stage_range(m.A, batch_at(a.cA, (long long)a.n + 1) + m.L0, m.L1 - m.L0 + 1);
        stage_range(m.BM, batch_at(a.cBM, 2LL * a.n) + 2 * m.L0, 2 * (m.L1 - m.L0));
    }
}

// On the finest level (f staged), in place over the staged cells (pairs 2J,
// 2J+1; L0 and L1 are even): f converted to G, then gs = G >> gsh rounded
// (the right-hand side in solution units) and, with gr, the restricted
// right-hand side of the coarse cells [J0, J1).  Below it gs keeps the staged
// G_l (m.gsh = gsh): the sweeps shift each value as they load it and the down
// pass restricts G where it forms tau, the same values without this pass.
__device__ void prepare_rhs(LevelSmem &m, const LevelArgs &a, int gsh, i64 *gr, int J0, int J1) {
    (void)a;
    const bool from_f = (m.gin == nullptr);
    m.gsh = from_f ? 0 : gsh;
    if (!from_f) return;
    const int kg = m.sc->Sg0;
    for (int J = (m.L0 >> 1) + (int)threadIdx.x; J < (m.L1 >> 1); J += (int)blockDim.x) {
        const int i = 2 * J - m.L0;
        i64 g0 = m.gs[i], g1 = m.gs[i + 1];
        if (from_f) {
            g0 = f64_to_fixed(__longlong_as_double(g0), kg);
            g1 = f64_to_fixed(__longlong_as_double(g1), kg);
        }
        if (gr && J >= J0 && J < J1) gr[J - J0] = restrict_rhs(g0, g1);
        m.gs[i] = shr_round(g0, gsh);
        m.gs[i + 1] = shr_round(g1, gsh);
    }
}

template <bool VC>
__device__ void smooth_range(LevelSmem &m, int n, int nu) {
    int lo = (m.L0 == 0) ? 0 : m.L0 + 1;
    int hi = (m.L1 == n) ? n : m.L1 - 1;
    const int Kb = VC ? m.sc->Kb : 0;
    for (int k = 0; k < nu; ++k) {
        const bool asc = (k & 1) == 0;
        if (VC) {
            if (m.gsh) lex_sweep_vc<kChunk, true>(m.u, m.gs, m.A, m.BM, m.L0, m.L0, lo, hi, n, asc, m.X, m.Y, Kb, m.gsh);
            else lex_sweep_vc<kChunk>(m.u, m.gs, m.A, m.BM, m.L0, m.L0, lo, hi, n, asc, m.X, m.Y, Kb);
        } else {
            if (m.gsh) lex_sweep<kChunk, false, true>(m.u, m.gs, m.L0, lo, hi, n, asc, m.X, m.gsh);
            else lex_sweep<kChunk>(m.u, m.gs, m.L0, lo, hi, n, asc, m.X);
        }
        if (lo > 0) ++lo;
        if (hi < n) --hi;
    }
}

__device__ __forceinline__ i64 coarse_reflect(const i64 *src, int j, int nc) {
    if (j < 0) return -src[-j - 1];
    if (j >= nc) return -src[2 * nc - 1 - j];
    return src[j];
}

template <bool FROM_PI, bool VC>
__global__ void __launch_bounds__(kSweepBlockMax, VC ? 1 : 2) level_down_kernel(LevelArgs a) {
    pdl_enter();

    extern __shared__ i64 smi[];
    const int s = blockIdx.x * a.tile;
    const int n = a.n, nc = n >> 1;
    LevelSmem m = level_smem(smi, s, a, FROM_PI);
    stage_g_async<VC>(m, a);
    const double *uf = batch_at(a.u_src_f64, n);
    if (FROM_PI) stage_coarse_async(m.c, m.usrc, m.C0, m.C1, nc);
    else if (uf) stage_range(m.u, uf + m.L0, m.L1 - m.L0);
    else stage_range(m.u, m.usrc + m.L0, m.L1 - m.L0);
    stage_wait();
    __syncthreads();
    const int J0 = s >> 1;
    prepare_rhs(m, a, 2 * a.l - 2, m.gr, J0, (s + a.tile) >> 1);
    if (uf) {           // the FP64 solution onto the fixed-point grid
        const int S = m.sc->S;
        for (int i = m.L0 + (int)threadIdx.x; i < m.L1; i += (int)blockDim.x)
            m.u[i - m.L0] = f64_to_fixed(__longlong_as_double(m.u[i - m.L0]), S);
    }
    if (FROM_PI) {
        fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
        __syncthreads();
        for (int J = (m.L0 >> 1) + (int)threadIdx.x; J < (m.L1 >> 1); J += (int)blockDim.x)
            fmg_interp2(m.c, m.C0, J, m.u[2 * J - m.L0], m.u[2 * J + 1 - m.L0]);
    }
    if (FROM_PI || !m.gin || uf) __syncthreads();    // (below the finest level without Pi nothing was written)
    smooth_range<VC>(m, n, a.nu);
    const i64 *u = m.u;
    const int tsh = 2 * a.l - 4;
    for (int J = J0 + (int)threadIdx.x; J < ((s + a.tile) >> 1); J += (int)blockDim.x) {
        int i0 = 2 * J - m.L0;
        i64 um2 = (J > 0) ? u[i0 - 2] : 0, um1 = (J > 0) ? u[i0 - 1] : 0;
        i64 u2 = (J < nc - 1) ? u[i0 + 2] : 0, u3 = (J < nc - 1) ? u[i0 + 3] : 0;
        m.ucout[J] = (u[i0] + u[i0 + 1]) >> 1;
        const i64 gr = m.gsh ? restrict_rhs(m.gs[i0], m.gs[i0 + 1]) : m.gr[J - J0];
        m.gcout[J] = VC ? tau_rhs_vc(gr, um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, tsh, m.A[i0], m.A[i0 + 2])
                     : (J > 0 && J < nc - 1) ? tau_rhs_interior(gr, um2, um1, u[i0], u[i0 + 1], u2, u3, tsh)
                                             : tau_rhs(gr, um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, tsh);
    }
    for (int i = s + (int)threadIdx.x; i < s + a.tile; i += (int)blockDim.x) m.uout[i] = u[i - m.L0];
}

// Up pass (Eq. 4): U_l += P (U_{l-1} - R U_l) (rounded to units), then nu sweeps.
template <bool VC>
__global__ void __launch_bounds__(kSweepBlockMax, VC ? 1 : 2) level_up_kernel(LevelArgs a) {
    pdl_enter();

    extern __shared__ i64 smi[];
    const int s = blockIdx.x * a.tile;
    const int n = a.n, nc = n >> 1;
    LevelSmem m = level_smem(smi, s, a, false);
    stage_g_async<VC>(m, a);
    stage_range(m.u, m.usrc + m.L0, m.L1 - m.L0);
    stage_coarse_async(m.c, m.ucsrc, m.C0, m.C1, nc);
    stage_wait();
    __syncthreads();
    prepare_rhs(m, a, 2 * a.l - 2, nullptr, 0, 0);
    // c_J = U_{l-1,J} - (R U_l)_J from the staged tile; no correction for the
    // coarse cells whose children lie outside it (they only reach the frozen
    // end cells L0 and L1-1; see the FP64 kernel)
    for (int j = max(m.C0, 0) + (int)threadIdx.x; j < min(m.C1, nc); j += (int)blockDim.x) {
        const int i0 = 2 * j;
        const bool inside = i0 >= m.L0 && i0 + 1 < m.L1;
        m.c[j - m.C0] = inside ? m.c[j - m.C0] - ((m.u[i0 - m.L0] + m.u[i0 + 1 - m.L0]) >> 1) : 0;
    }
    __syncthreads();
    // the ghost coarse cells beyond the walls by odd reflection, read in place
    for (int i = m.L0 + (int)threadIdx.x; i < m.L1; i += (int)blockDim.x) {
        int J = i >> 1, nb = (i & 1) ? J + 1 : J - 1;
        const i64 cn = (nb < 0) ? -m.c[-m.C0] : ((nb >= nc) ? -m.c[nc - 1 - m.C0] : m.c[nb - m.C0]);
        m.u[i - m.L0] += (3 * m.c[J - m.C0] + cn + 2) >> 2;
    }
    __syncthreads();
    smooth_range<VC>(m, n, a.nu);
    const i64 *u = m.u;
    if (m.uout64) {
        const int S = m.sc->S;
        for (int i = s + (int)threadIdx.x; i < s + a.tile; i += (int)blockDim.x)
            m.uout64[i] = fixed_to_f64(u[i - m.L0], S);
    } else {
        for (int i = s + (int)threadIdx.x; i < s + a.tile; i += (int)blockDim.x) m.uout[i] = u[i - m.L0];
    }
}

// --------------------------------------------------------------------------
// Chains of stored-level passes (-u'' = f): the down passes of k consecutive
// levels, or their up passes, in one launch.  On the latency-bound small
// levels a pass costs a launch, a grid-wide dependency and a staging round
// more than its few sweeps; a chain keeps the k levels of a tile in shared
// memory instead.  Each level of a chain is a tile of the ordinary pass with
// a wider halo where the next level of the chain needs more exact cells: the
// same sweeps over ranges that cover the ordinary tile's, so every cell
// written is the same bits as the separate passes give.
// --------------------------------------------------------------------------
constexpr int kChainMax = 4;

struct ChainArgs {
    int k;                     // levels in the chain (2 .. kChainMax)
    int l;                     // down: the first (finest) level; up: the first (coarsest) level
    int tile;                  // owned cells of a block on the chain's finest level
    int H;                     // halo of one level's sweeps (112 nu)
    int nu;
    int off[kChainMax], len[kChainMax];   // shared memory of chain level i: U at off[i], G at off[i] + len[i]
    int off_c, off_x;          // coarse cells of an up step; chunk carries
    const Scale *sc;
    const i64 *u_src;          // down: the first level's iterate
    const i64 *uc_src;         // up: the corrected level below the chain
    const i64 *u_in[kChainMax];   // up: each level's iterate after its down pass
    const i64 *g[kChainMax];   // G of each level (down: only g[0] is read)
    i64 *u_out[kChainMax];     // each level after its sweeps (owned cells)
    i64 *g_out[kChainMax];     // down: G (tau right-hand side) of the level below chain level i (owned cells)
    i64 *uc_out;               // down: U of the level below the chain (restriction, owned cells)
};

__device__ __forceinline__ LevelSmem chain_level_smem(i64 *smi, const ChainArgs &a, int i, int l, int L0, int L1) {
    LevelSmem m;
    m.u = smi + a.off[i];
    m.gs = m.u + a.len[i];
    m.c = smi + a.off_c;
    m.X = smi + a.off_x;
    m.gr = nullptr;
    m.Y = nullptr;
    m.A = nullptr;
    m.BM = nullptr;
    m.gsh = 2 * l - 2;         // G below the finest level, shifted by the sweeps
    m.L0 = L0;
    m.L1 = L1;
    m.C0 = (L0 >> 1) - 2;
    m.C1 = ((L1 - 1) >> 1) + 3;
    m.sc = a.sc + blockIdx.y;
    return m;
}

// Down chain: chain level i is level l - i with owned cells [s >> i, (s + T) >> i)
// and halo h_i, h_{k-1} = H, h_i = 2 h_{i+1} + H: after its sweeps the cells
// the next level's halo is restricted from are exact (a tile of halo H gives
// exact values H cells in, the tau stencil included).  Level i's restriction
// and tau fill level i+1's whole held range in shared memory; the owned
// coarse cells also go to global memory (G of every level below, for the up
// passes; U of the level below the chain).
__global__ void __launch_bounds__(kSweepBlockMax, 2) level_down_chain_kernel(const __grid_constant__ ChainArgs a) {
    pdl_enter();
    extern __shared__ i64 smi[];
    int h[kChainMax];
    h[a.k - 1] = a.H;
    for (int i = a.k - 2; i >= 0; --i) h[i] = 2 * h[i + 1] + a.H;
    const int s0 = blockIdx.x * a.tile;
    {
        const int n = 1 << a.l;
        const int L0 = max(0, s0 - h[0]), L1 = min(n, s0 + a.tile + h[0]);
        stage_range(smi + a.off[0], batch_at(a.u_src, n) + L0, L1 - L0);
        stage_range(smi + a.off[0] + a.len[0], batch_at(a.g[0], n) + L0, L1 - L0);
        stage_wait();
        __syncthreads();
    }
    for (int i = 0; i < a.k; ++i) {
        const int l = a.l - i, n = 1 << l, nc = n >> 1;
        const int s = s0 >> i, T = a.tile >> i;
        LevelSmem m = chain_level_smem(smi, a, i, l, max(0, s - h[i]), min(n, s + T + h[i]));
        smooth_range<false>(m, n, a.nu);
        const i64 *u = m.u;
        i64 *uo = batch_at(a.u_out[i], n);
        for (int q = s + (int)threadIdx.x; q < s + T; q += (int)blockDim.x) uo[q] = u[q - m.L0];
        // the coarse cells of the next chain level's held range (or, after the
        // last level, the owned ones)
        const bool last = (i == a.k - 1);
        const int Jo0 = s >> 1, Jo1 = (s + T) >> 1;
        const int Jlo = last ? Jo0 : max(0, Jo0 - h[i + 1]), Jhi = last ? Jo1 : min(nc, Jo1 + h[i + 1]);
        i64 *un = last ? nullptr : smi + a.off[i + 1];
        i64 *gn = last ? nullptr : un + a.len[i + 1];
        i64 *gco = batch_at(a.g_out[i], nc);
        i64 *uco = last ? batch_at(a.uc_out, nc) : nullptr;
        const int tsh = 2 * l - 4;
        for (int J = Jlo + (int)threadIdx.x; J < Jhi; J += (int)blockDim.x) {
            const int i0 = 2 * J - m.L0;
            const i64 um2 = (J > 0) ? u[i0 - 2] : 0, um1 = (J > 0) ? u[i0 - 1] : 0;
            const i64 u2 = (J < nc - 1) ? u[i0 + 2] : 0, u3 = (J < nc - 1) ? u[i0 + 3] : 0;
            const i64 ucv = (u[i0] + u[i0 + 1]) >> 1;
            const i64 gr = restrict_rhs(m.gs[i0], m.gs[i0 + 1]);
            const i64 gcv = (J > 0 && J < nc - 1) ? tau_rhs_interior(gr, um2, um1, u[i0], u[i0 + 1], u2, u3, tsh)
                                                  : tau_rhs(gr, um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, tsh);
            if (!last) {
                un[J - Jlo] = ucv;
                gn[J - Jlo] = gcv;
            }
            if (J >= Jo0 && J < Jo1) {
                gco[J] = gcv;
                if (last) uco[J] = ucv;
            }
        }
        __syncthreads();
    }
}

// Up chain: chain level i is level l + i, bottom up; the last (finest) level
// is the ordinary up tile [s - H, s + T + H) of the block's T cells, and each
// level below holds the coarse range that the level above interpolates from
// plus a halo H, so that range comes out exact.  Every level's held range is
// staged at once; the coarse cells of level i's correction are level i-1's
// result in shared memory (the corrected level below the chain from global
// memory for i = 0).  Each level writes its owned cells: the block's T cells
// of the finest level, scaled by 2^-(k-1-i) on chain level i.
__global__ void __launch_bounds__(kSweepBlockMax, 2) level_up_chain_kernel(const __grid_constant__ ChainArgs a) {
    pdl_enter();
    extern __shared__ i64 smi[];
    int L0[kChainMax], L1[kChainMax];
    const int top = a.k - 1;
    const int s0 = blockIdx.x * a.tile;
    L0[top] = max(0, s0 - a.H);
    L1[top] = min(1 << (a.l + top), s0 + a.tile + a.H);
    for (int i = top - 1; i >= 0; --i) {
        const int n = 1 << (a.l + i);
        const int C0 = max(0, (L0[i + 1] >> 1) - 2), C1 = min(n, ((L1[i + 1] - 1) >> 1) + 3);
        L0[i] = max(0, C0 - a.H);
        L1[i] = min(n, C1 + a.H);
    }
    for (int i = 0; i < a.k; ++i) {
        const int n = 1 << (a.l + i);
        stage_range(smi + a.off[i], batch_at(a.u_in[i], n) + L0[i], L1[i] - L0[i]);
        stage_range(smi + a.off[i] + a.len[i], batch_at(a.g[i], n) + L0[i], L1[i] - L0[i]);
    }
    {
        const int nc = 1 << (a.l - 1);
        const int C0 = (L0[0] >> 1) - 2, C1 = ((L1[0] - 1) >> 1) + 3;
        stage_coarse_async(smi + a.off_c, batch_at(a.uc_src, nc), C0, C1, nc);
    }
    stage_wait();
    __syncthreads();
    for (int i = 0; i < a.k; ++i) {
        const int l = a.l + i, n = 1 << l, nc = n >> 1;
        LevelSmem m = chain_level_smem(smi, a, i, l, L0[i], L1[i]);
        const i64 *prev = (i > 0) ? smi + a.off[i - 1] : nullptr;   // level l-1, held from L0[i-1]
        // c_J = U_{l-1,J} - (R U_l)_J, 0 for the coarse cells whose children lie
        // outside the held range (they reach only its frozen end cells)
        for (int j = max(m.C0, 0) + (int)threadIdx.x; j < min(m.C1, nc); j += (int)blockDim.x) {
            const int i0 = 2 * j;
            const bool inside = i0 >= m.L0 && i0 + 1 < m.L1;
            const i64 uc = prev ? prev[j - L0[i - 1]] : m.c[j - m.C0];
            m.c[j - m.C0] = inside ? uc - ((m.u[i0 - m.L0] + m.u[i0 + 1 - m.L0]) >> 1) : 0;
        }
        __syncthreads();
        for (int q = m.L0 + (int)threadIdx.x; q < m.L1; q += (int)blockDim.x) {
            const int J = q >> 1, nb = (q & 1) ? J + 1 : J - 1;
            const i64 cn = (nb < 0) ? -m.c[-m.C0] : ((nb >= nc) ? -m.c[nc - 1 - m.C0] : m.c[nb - m.C0]);
            m.u[q - m.L0] += (3 * m.c[J - m.C0] + cn + 2) >> 2;
        }
        __syncthreads();
        smooth_range<false>(m, n, a.nu);
        const int sh = top - i;
        const int s = s0 >> sh, T = a.tile >> sh;
        i64 *uo = batch_at(a.u_out[i], n);
        for (int q = s + (int)threadIdx.x; q < s + T; q += (int)blockDim.x) uo[q] = m.u[q - m.L0];
    }
}

// --------------------------------------------------------------------------
// SR level (Fig. 3): one block per segment.
// --------------------------------------------------------------------------
struct SegArgs {
    int M, n, W, b, nu;
    int maxlen, maxc, maxch;
    int seg0;                  // post-leg: first segment (block x handles segment seg0 + x)
    int local_tau;             // pre-leg: tau of the edge coarse cells from the own patch (no seam pass)
    const Scale *sc;
    const double *f;           // the finest level's rhs
    const i64 *g_in;           // SR level below the finest: its rhs G_M (then f is unused)
    const i64 *u_in;           // pre-leg of an SR level below the top: its assembled iterate (no Pi)
    const double *u_in_f64;    // pre-leg of a further V-cycle: the current FP64 fine solution (no Pi)
    const i64 *uc_src;
    i64 *uc_out, *gc_out, *seam;
    i64 *u_out_fx;             // post-leg of an SR level below the finest: U of the level
    double *u_out;             // post-leg: FP64 solution of segments seg0.. (NULL: not written)
    const double *u_ref;       // post-leg: reference for the functionals (NULL: none)
    double *fpart;             // post-leg: kNumFunc partials per segment (NULL: no functionals)
    const u64 *cA, *cBM;       // variable coefficient: the level's A (faces) and multipliers (cells)
    // post-leg option FAS recompute, as in the FP64 SegArgs (the second coarse
    // array of the post-leg is gr, which the post-leg does not otherwise use)
    i64 *u_old_out, *edge_out;
    const i64 *uc_corr, *uhat, *edge_in;
    int nu_pre;
};

// Shared memory as LevelSmem: u, gs, c, X, gr (2 maxlen + 2 maxc + maxch words),
// and for the variable coefficient A, BM and Y (3 maxlen + 1 + maxch more).
struct SegSmem {
    i64 *u, *gs, *c, *X, *gr, *Y;
    u64 *A, *BM;
    int e0, e1, lo, hi, C0, C1;
};

// (The arrays of problem blockIdx.y are formed where they are used, see
// batch_at, so that their pointers do not stay live across the sweeps.)

__device__ __forceinline__ SegSmem seg_smem(i64 *sm, const SegArgs &a, int s) {
    SegSmem m;
    m.e0 = max(0, s - a.b);
    m.e1 = min(a.n, s + a.W + a.b);
    m.lo = (m.e0 > 0) ? m.e0 - 1 : 0;
    m.hi = (m.e1 < a.n) ? m.e1 + 1 : a.n;
    m.C0 = (m.lo >> 1) - 2;
    m.C1 = ((m.hi - 1) >> 1) + 3;
    m.u = sm;
    m.gs = m.u + a.maxlen;
    m.c = m.gs + a.maxlen;
    m.X = m.c + a.maxc;
    m.gr = m.X + a.maxch;
    m.A = (u64 *)(m.gr + a.maxc);
    m.BM = m.A + a.maxlen + 1;
    m.Y = (i64 *)(m.BM + 2 * a.maxlen);
    return m;
}

// Stage the patch [lo, hi) of an SR level M: the iterate Pi U_{M-1} (or, with
// u_in, the assembled iterate of a level below the top, in the down leg) and
// the right-hand side gs = G >> (2M-2) in solution units, G converted from f
// on the finest level or read from g_in below it; with gr, also the restricted
// right-hand side of the segment's coarse cells [J0, J1).  The staged range
// may start at an odd cell, so pairs are clipped to it.  With kacz, the first
// Kaczmarz pass of the post-leg (Fig. 5) is applied to the pairs inside the
// extended patch as they are interpolated (the same arithmetic as the
// separate pass, without its extra sweep over shared memory); the return value
// says whether that happened (not when the iterate is staged instead of Pi).
template <bool VC>
__device__ bool seg_load(SegSmem &m, const SegArgs &a, i64 *gr, int J0, int J1, bool kacz = false) {
    const int nc = a.n >> 1, kg = (a.sc + blockIdx.y)->Sg0, gsh = 2 * a.M - 2;
    const bool from_f = (a.g_in == nullptr);
    if (VC) {
        stage_range(m.A, batch_at(a.cA, (long long)a.n + 1) + m.lo, m.hi - m.lo + 1);
        stage_range(m.BM, batch_at(a.cBM, 2LL * a.n) + 2 * m.lo, 2 * (m.hi - m.lo));
    }
    if (a.u_in) stage_range(m.u, batch_at(a.u_in, a.n) + m.lo, m.hi - m.lo);
    else if (a.u_in_f64) stage_range(m.u, batch_at(a.u_in_f64, a.n) + m.lo, m.hi - m.lo);
    else stage_coarse_async(m.c, batch_at(a.uc_src, nc), m.C0, m.C1, nc);
    if (from_f) stage_range(m.gs, batch_at(a.f, a.n) + m.lo, m.hi - m.lo);
    else stage_range(m.gs, batch_at(a.g_in, a.n) + m.lo, m.hi - m.lo);
    stage_wait();
    __syncthreads();
    if (!a.u_in && !a.u_in_f64) fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
    const int S = (a.sc + blockIdx.y)->S;
    for (int J = (m.lo >> 1) + (int)threadIdx.x; 2 * J < m.hi; J += (int)blockDim.x) {
        const int i0 = 2 * J;
        const bool in0 = i0 >= m.lo, in1 = i0 + 1 < m.hi;
        const i64 f0 = m.gs[max(i0 - m.lo, 0)], f1 = m.gs[min(i0 + 1 - m.lo, m.hi - 1 - m.lo)];
        const i64 g0 = from_f ? f64_to_fixed(__longlong_as_double(f0), kg) : f0;
        const i64 g1 = from_f ? f64_to_fixed(__longlong_as_double(f1), kg) : f1;
        if (gr && J >= J0 && J < J1) gr[J - J0] = restrict_rhs(g0, g1);
        if (in0) m.gs[i0 - m.lo] = shr_round(g0, gsh);
        if (in1) m.gs[i0 + 1 - m.lo] = shr_round(g1, gsh);
        if (a.u_in_f64) {   // the FP64 solution onto the fixed-point grid
            if (in0) m.u[i0 - m.lo] = f64_to_fixed(__longlong_as_double(m.u[i0 - m.lo]), S);
            if (in1) m.u[i0 + 1 - m.lo] = f64_to_fixed(__longlong_as_double(m.u[i0 + 1 - m.lo]), S);
        }
    }
    __syncthreads();
    if (a.u_in || a.u_in_f64) return false;
    for (int J = (m.lo >> 1) + (int)threadIdx.x; 2 * J < m.hi; J += (int)blockDim.x) {
        i64 l, r;
        fmg_interp2(m.c, m.C0, J, l, r);
        if (kacz && 2 * J >= m.e0 && 2 * J + 1 < m.e1) {
            const i64 k = m.c[J - m.C0] - ((l + r) >> 1);
            l += k;
            r += k;
        }
        if (2 * J >= m.lo) m.u[2 * J - m.lo] = l;
        if (2 * J + 1 < m.hi) m.u[2 * J + 1 - m.lo] = r;
    }
    __syncthreads();
    return kacz;
}

template <bool VC>
__global__ void __launch_bounds__(kSweepBlockMax, VC ? 1 : 2) sr_pre_kernel(SegArgs a) {
    pdl_enter();
    extern __shared__ i64 smi[];
    const int s = blockIdx.x * a.W;
    const int n = a.n, nc = n >> 1;
    SegSmem m = seg_smem(smi, a, s);
    const int J0 = s >> 1, J1 = (s + a.W) >> 1;
    seg_load<VC>(m, a, m.gr, J0, J1);
    if (a.u_old_out) {        // the interpolated iterate on the segment's coarse cells (post-leg recompute)
        i64 *uo = batch_at(a.u_old_out, nc);
        for (int J = J0 + (int)threadIdx.x; J < J1; J += (int)blockDim.x) uo[J] = m.c[J - m.C0];
    }
    const int tsh = 2 * a.M - 4;
    const int Kb = VC ? (a.sc + blockIdx.y)->Kb : 0;
    for (int k = 0; k < a.nu; ++k) {
        if (VC) lex_sweep_vc<kChunk>(m.u, m.gs, m.A, m.BM, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y, Kb);
        else lex_sweep<kChunk>(m.u, m.gs, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X);
    }
    if (a.edge_out) {         // the pre-smoothed interior cells the neighbours' patches read
        const int ne = a.b + 1;
        i64 *eo = batch_at(a.edge_out, (long long)(n / a.W) * 2 * ne) + (size_t)blockIdx.x * 2 * ne;
        for (int k = threadIdx.x; k < ne; k += blockDim.x) {
            eo[k] = m.u[s + k - m.lo];
            eo[ne + k] = m.u[s + a.W - ne + k - m.lo];
        }
    }
    const i64 *u = m.u;
    i64 *uc_out = batch_at(a.uc_out, nc), *gc_out = batch_at(a.gc_out, nc);
    for (int J = J0 + (int)threadIdx.x; J < J1; J += (int)blockDim.x) {
        int i0 = 2 * J - m.lo;
        uc_out[J] = (u[i0] + u[i0 + 1]) >> 1;
        bool edge = !a.local_tau && ((J == J0 && J > 0) || (J == J1 - 1 && J < nc - 1));
        if (!edge) {
            i64 um2 = (J > 0) ? u[i0 - 2] : 0, um1 = (J > 0) ? u[i0 - 1] : 0;
            i64 u2 = (J < nc - 1) ? u[i0 + 2] : 0, u3 = (J < nc - 1) ? u[i0 + 3] : 0;
            gc_out[J] = VC ? tau_rhs_vc(m.gr[J - J0], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, tsh, m.A[i0],
                                        m.A[i0 + 2])
                        : (J > 0 && J < nc - 1) ? tau_rhs_interior(m.gr[J - J0], um2, um1, u[i0], u[i0 + 1], u2, u3, tsh)
                                                : tau_rhs(m.gr[J - J0], um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, tsh);
        }
    }
    if (threadIdx.x < 6) {
        int k = threadIdx.x;
        int i = (k < 3) ? s + k : s + a.W - 6 + k;
        batch_at(a.seam, 6LL * (n / a.W))[(size_t)blockIdx.x * 6 + k] = u[i - m.lo];
    }
}

// tau rhs at the two coarse cells of each interior segment boundary from the
// assembled fine values (seams) and the restricted solution.
template <bool VC>
__global__ void seam_tau_kernel(SegArgs a, int nseg) {
    pdl_enter();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nseg - 1) return;
    const int s = (k + 1) * a.W;
    const int kg = (a.sc + blockIdx.y)->Sg0, tsh = 2 * a.M - 4;
    const i64 *seam = batch_at(a.seam, 6LL * nseg);
    const double *f = batch_at(a.f, a.n);
    const i64 *gl = a.g_in ? batch_at(a.g_in, a.n) : nullptr;      // G of a level below the finest
    i64 *uc_out = batch_at(a.uc_out, a.n / 2), *gc_out = batch_at(a.gc_out, a.n / 2);
    const i64 *L = seam + (size_t)k * 6, *R = seam + (size_t)(k + 1) * 6;
    const i64 f3 = L[3], f2 = L[4], f1 = L[5], p0 = R[0], p1 = R[1], p2 = R[2];
    const int J = (s >> 1) - 1;
    const i64 hm1 = uc_out[J - 1], h0 = uc_out[J], h1 = uc_out[J + 1], h2 = uc_out[J + 2];
    // variable coefficient: the fine faces s - 2, s, s + 2 (coarse faces J, J + 1, J + 2)
    const u64 *cA = VC ? batch_at(a.cA, (long long)a.n + 1) : nullptr;
    {
        i64 g0 = gl ? gl[2 * J] : f64_to_fixed(f[2 * J], kg), g1 = gl ? gl[2 * J + 1] : f64_to_fixed(f[2 * J + 1], kg);
        if (VC) {
            const i64 dl = (h0 - hm1) - 2 * (f2 - f3), dr = (h1 - h0) - 2 * (p0 - f1);
            gc_out[J] = ((g0 + g1 + 1) >> 1) +
                        s128_diff_shr_round(mul_s128(cA[s - 2], dl), mul_s128(cA[s], dr), kSaVc - tsh);
        } else {
            i64 tau = ((h0 - hm1) - (h1 - h0)) - 2 * ((f2 - f3) - (p0 - f1));
            gc_out[J] = ((g0 + g1 + 1) >> 1) + tau * (1LL << tsh);
        }
    }
    {
        const int J2 = J + 1;
        i64 g0 = gl ? gl[2 * J2] : f64_to_fixed(f[2 * J2], kg), g1 = gl ? gl[2 * J2 + 1] : f64_to_fixed(f[2 * J2 + 1], kg);
        if (VC) {
            const i64 dl = (h1 - h0) - 2 * (p0 - f1), dr = (h2 - h1) - 2 * (p2 - p1);
            gc_out[J2] = ((g0 + g1 + 1) >> 1) +
                         s128_diff_shr_round(mul_s128(cA[s], dl), mul_s128(cA[s + 2], dr), kSaVc - tsh);
        } else {
            i64 tau = ((h1 - h0) - (h2 - h1)) - 2 * ((p0 - f1) - (p2 - p1));
            gc_out[J2] = ((g0 + g1 + 1) >> 1) + tau * (1LL << tsh);
        }
    }
}

// Sum of squares of non-negative fixed-point values A < 2^59 in integers:
// V = A >> 8 split as V = 2^26 va + vb, V^2 = 2^52 va^2 + 2^27 va vb + vb^2 in
// three 64-bit sums.  A thread adds at most 16 values (va^2 < 2^50 each);
// norm() carries q0 into q1 and q1 into q2 (weights 2^27 and 2^25 apart), after
// which 512 threads' sums stay below 2^63.  A^2 ~ 2^16 V^2: dropping 8 of A's
// bits moves a square by at most 2^-50 of the largest.  value(S) is the sum of
// (A 2^-S)^2 as a double.
struct FxSquares {
    u64 q0 = 0, q1 = 0, q2 = 0;
    __device__ __forceinline__ void add(u64 A) {
        const u64 V = A >> 8, va = V >> 26, vb = V & 0x3ffffffULL;
        q2 += va * va;
        q1 += va * vb;
        q0 += vb * vb;
    }
    __device__ __forceinline__ void norm() {
        q1 += q0 >> 27;
        q0 &= (1ULL << 27) - 1;
        q2 += q1 >> 25;
        q1 &= (1ULL << 25) - 1;
    }
    __device__ __forceinline__ double value(int S) const {
        return scale2(fma((double)q2, 4503599627370496.0, fma((double)q1, 134217728.0, (double)q0)), 16 - 2 * S);
    }
};

// The functional state of one thread in integers: sum U in 128 bits (hi, lo),
// max |U|, the squares; against the reference, max |D| and the squares of D;
// e3, e4 the FP64 terms of references beyond the integer grid's range.
struct FxFunc {
    u64 lo = 0, mx = 0, mxd = 0;
    i64 hi = 0;
    FxSquares su, sd;
    double e3 = 0.0, e4 = 0.0;
};

// Warp butterfly over the ten integer words of FxFunc (128-bit add with carry,
// maxima, limb sums): exact, the same in every lane.
__device__ __forceinline__ void fx_warp_reduce(u64 v[10]) {
    for (int o = 16; o > 0; o >>= 1) {
        u64 y[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) y[k] = __shfl_xor_sync(0xffffffffu, v[k], o);
        const u64 lo = v[0] + y[0];
        v[1] = v[1] + y[1] + (lo < v[0] ? 1ULL : 0ULL);
        v[0] = lo;
        v[2] = y[2] > v[2] ? y[2] : v[2];
        v[6] = y[6] > v[6] ? y[6] : v[6];
        v[3] += y[3]; v[4] += y[4]; v[5] += y[5];
        v[7] += y[7]; v[8] += y[8]; v[9] += y[9];
    }
}

// Reduce the block's FxFunc in integers (FP64 only for e3, e4, through the
// integer-grid warp sums) and write the segment's kNumFunc partials from
// thread 0.  Every thread of the block calls it once; blockDim.x <= 512.
__device__ __forceinline__ void fx_block_functionals(FxFunc &t, int S, double *dst) {
    __shared__ u64 red[10][16];
    __shared__ double red64[2][16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    t.su.norm();
    t.sd.norm();
    u64 v[10] = {t.lo, (u64)t.hi, t.mx, t.su.q0, t.su.q1, t.su.q2, t.mxd, t.sd.q0, t.sd.q1, t.sd.q2};
    fx_warp_reduce(v);
    const double w3 = warp_sum(t.e3), w4 = warp_max_nonneg(t.e4);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 10; ++k) red[k][w] = v[k];
        red64[0][w] = w3;
        red64[1][w] = w4;
    }
    __syncthreads();
    if (w != 0) return;
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = lane < nw ? red[k][lane] : 0ULL;
    fx_warp_reduce(v);
    const double e3 = warp_sum(lane < nw ? red64[0][lane] : 0.0);
    const double e4 = warp_max_nonneg(lane < nw ? red64[1][lane] : 0.0);
    if (lane != 0) return;
    FxSquares su, sd;
    su.q0 = v[3]; su.q1 = v[4]; su.q2 = v[5];
    sd.q0 = v[7]; sd.q1 = v[8]; sd.q2 = v[9];
    dst[0] = scale2(fma((double)(i64)v[1], 18446744073709551616.0, (double)v[0]), -S);   // hi 2^64 + lo
    dst[1] = su.value(S);
    dst[2] = scale2((double)v[2], -S);
    dst[3] = e3 + sd.value(S);
    dst[4] = fmax(e4, scale2((double)v[6], -S));
}

// K6 in fixed point; output and functionals as in the FP64 kernel.
template <bool VC>
__global__ void __launch_bounds__(kSweepBlockMax, VC ? 1 : 2) sr_post_kernel(SegArgs a) {
    pdl_enter();
    extern __shared__ i64 smi[];
    const int s = (a.seg0 + (int)blockIdx.x) * a.W;
    const int n = a.n;
    SegSmem m = seg_smem(smi, a, s);
    const bool rcm = a.uc_corr != nullptr;          // post-leg option FAS recompute
    const bool first_done = seg_load<VC>(m, a, nullptr, 0, 0, !rcm);
    const int Kb = VC ? (a.sc + blockIdx.y)->Kb : 0;
    i64 *p = m.u;
    if (rcm) {
        // the pre-smoothed patch as the pre-leg formed it ...
        for (int k = 0; k < a.nu_pre; ++k) {
            if (VC) lex_sweep_vc<kChunk>(p, m.gs, m.A, m.BM, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y, Kb);
            else lex_sweep<kChunk>(p, m.gs, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X);
        }
        // ... with the assembled values in its buffer and frozen cells ...
        const int ne = a.b + 1, seg = a.seg0 + (int)blockIdx.x, nseg = n / a.W;
        const i64 *ei = batch_at(a.edge_in, (long long)nseg * 2 * ne);
        for (int i = m.lo + (int)threadIdx.x; i < s; i += (int)blockDim.x)
            p[i - m.lo] = ei[(size_t)(seg - 1) * 2 * ne + ne + (i - (s - ne))];
        for (int i = s + a.W + (int)threadIdx.x; i < m.hi; i += (int)blockDim.x)
            p[i - m.lo] = ei[(size_t)(seg + 1) * 2 * ne + (i - (s + a.W))];
        // ... corrected by Eq. 4: U += P (U_{M-1} - R Ubar), rounded to units ...
        const int nc = n >> 1;
        stage_coarse_async(m.c, batch_at(a.uc_corr, nc), m.C0, m.C1, nc);
        stage_coarse_async(m.gr, batch_at(a.uhat, nc), m.C0, m.C1, nc);
        stage_wait();
        __syncthreads();
        fill_coarse_ghosts(m.c, m.C0, m.C1, nc);
        fill_coarse_ghosts(m.gr, m.C0, m.C1, nc);
        __syncthreads();
        for (int j = m.C0 + (int)threadIdx.x; j < m.C1; j += (int)blockDim.x) m.c[j - m.C0] -= m.gr[j - m.C0];
        __syncthreads();
        for (int i = m.lo + (int)threadIdx.x; i < m.hi; i += (int)blockDim.x) {
            const int J = i >> 1, nb = (i & 1) ? J + 1 : J - 1;
            p[i - m.lo] += (3 * m.c[J - m.C0] + m.c[nb - m.C0] + 2) >> 2;
        }
        __syncthreads();
    }
    for (int k = 0; k < a.nu; ++k) {
        if (!rcm && (k > 0 || !first_done)) {   // Kaczmarz (Fig. 5), not in the FAS recompute
            for (int J = (m.e0 >> 1) + (int)threadIdx.x; J < (m.e1 >> 1); J += (int)blockDim.x) {
                int i0 = 2 * J - m.lo;
                i64 r = m.c[J - m.C0] - ((p[i0] + p[i0 + 1]) >> 1);
                p[i0] += r;
                p[i0 + 1] += r;
            }
            __syncthreads();
        }
        if (VC) lex_sweep_vc<kChunk>(p, m.gs, m.A, m.BM, m.lo, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X, m.Y, Kb);
        else lex_sweep<kChunk>(p, m.gs, m.lo, m.e0, m.e1, n, (k & 1) == 0, m.X);
    }
    const int S = (a.sc + blockIdx.y)->S;
    const long long s0 = (long long)a.seg0 * a.W;     // first cell of the output
    double *u_out = a.u_out ? batch_at(a.u_out, (long long)gridDim.x * a.W) : nullptr;
    if (u_out && ((uintptr_t)u_out & 15) == 0) {      // pairs of cells, 16-byte stores (W is even)
        double2 *o2 = reinterpret_cast<double2 *>(u_out + (s - s0));
        for (int j = (int)threadIdx.x; j < (a.W >> 1); j += (int)blockDim.x) {
            const int i = s + 2 * j - m.lo;
            o2[j] = make_double2(fixed_to_f64(p[i], S), fixed_to_f64(p[i + 1], S));
        }
    } else if (u_out) {
        for (int i = s + (int)threadIdx.x; i < s + a.W; i += (int)blockDim.x)
            u_out[i - s0] = fixed_to_f64(p[i - m.lo], S);
    }
    if (a.u_out_fx) {
        i64 *uo = batch_at(a.u_out_fx, a.n);
        for (int i = s + (int)threadIdx.x; i < s + a.W; i += (int)blockDim.x) uo[i] = p[i - m.lo];
    }
    if (a.fpart) {
        // The functionals in integer arithmetic (FxFunc): against a reference r,
        // D = U - round(r 2^S) exactly on the fixed-point grid; a reference beyond
        // that grid's range (|r| 2^S >= 2^59, or not finite) or a |D| >= 2^59
        // takes FP64.
        const bool ref = a.u_ref != nullptr;
        if (ref) {   // the reference of the interior into the rhs array, which the sweeps are done with
            __syncthreads();
            stage_range(m.gs + (s - m.lo), batch_at(a.u_ref, a.n) + s, a.W);
            stage_wait();
            __syncthreads();
        }
        FxFunc t;
        for (int i = s + (int)threadIdx.x; i < s + a.W; i += (int)blockDim.x) {
            const i64 U = p[i - m.lo];
            t.lo += (u64)U;
            t.hi += (U >> 63) + (t.lo < (u64)U ? 1 : 0);
            const u64 A = (u64)(U < 0 ? -U : U);
            t.mx = A > t.mx ? A : t.mx;
            t.su.add(A);
            if (ref) {
                const double r = __longlong_as_double(m.gs[i - m.lo]);
                const int e = (int)((__double_as_longlong(r) >> 52) & 0x7ff) - 1023;   // |r| < 2^(e+1)
                const i64 D = (e + S <= 57) ? U - f64_to_fixed(r, S) : 0;
                const u64 AD = (u64)(D < 0 ? -D : D);
                if (e + S <= 57 && AD < (1ULL << 59)) {
                    t.mxd = AD > t.mxd ? AD : t.mxd;
                    t.sd.add(AD);
                } else {
                    const double d = fixed_to_f64(U, S) - r;
                    t.e3 = fma(d, d, t.e3);
                    t.e4 = fmax(t.e4, fabs(d));
                }
            }
        }
        fx_block_functionals(t, S, batch_at(a.fpart, (long long)gridDim.x * kNumFunc) + (long long)blockIdx.x * kNumFunc);
    }
}

// --------------------------------------------------------------------------
// Coarse tail (one block, levels M0..Mc in shared memory); the coarsest
// level is solved in FP64 with the dense inverse.
// --------------------------------------------------------------------------
struct TailArgs {
    int M0, Mc, nu1, nu2, mode;
    const Scale *sc;
    const i64 *u_in;
    const i64 *g_in;           // G_Mc, or NULL to read f
    const double *f;
    i64 *u_out;
    double *u_out_f64;         // whole problem in the tail: the FP64 solution
    const double *Ainv;
    // variable coefficient: per level, A (faces) and the multipliers (cells), and the
    // FP64 face coefficients of the coarsest level (its Thomas solve)
    const u64 *cA[32];
    const u64 *cBM[32];
    const double *coef0;
};

struct TailSmem {
    i64 *u, *g, *S, *X, *Y;
    int M0, Kb;
    const u64 *const *cA;
    const u64 *const *cBM;
    __device__ int off(int l) const { return (1 << l) - (1 << M0); }
    // this problem's coefficient words of level l
    __device__ const u64 *A(int l) const { return batch_at(cA[l], (1LL << l) + 1); }
    __device__ const u64 *BM(int l) const { return batch_at(cBM[l], 2LL << l); }
};

// nu sweeps of level l on G_l directly (the sweep shifts it into solution units)
template <bool VC>
__device__ void tail_smooth(TailSmem &m, int l, int nu) {
    const int n = 1 << l;
    i64 *u = m.u + m.off(l);
    const i64 *g = m.g + m.off(l);
    for (int k = 0; k < nu; ++k) {
        if (VC) lex_sweep_vc<kChunk, true>(u, g, m.A(l), m.BM(l), 0, 0, 0, n, n, (k & 1) == 0, m.X, m.Y, m.Kb,
                                           2 * l - 2);
        else lex_sweep<kChunk, true, true>(u, g, 0, 0, n, n, (k & 1) == 0, m.X, 2 * l - 2);
    }
}

template <bool VC>
__device__ void tail_down(TailSmem &m, int l, int nu) {
    tail_smooth<VC>(m, l, nu);
    const int nc = 1 << (l - 1);
    const i64 *u = m.u + m.off(l), *g = m.g + m.off(l);
    i64 *uc = m.u + m.off(l - 1), *gc = m.g + m.off(l - 1);
    for (int J = threadIdx.x; J < nc; J += blockDim.x) {
        int i0 = 2 * J;
        i64 um2 = (J > 0) ? u[i0 - 2] : 0, um1 = (J > 0) ? u[i0 - 1] : 0;
        i64 u2 = (J < nc - 1) ? u[i0 + 2] : 0, u3 = (J < nc - 1) ? u[i0 + 3] : 0;
        uc[J] = (u[i0] + u[i0 + 1]) >> 1;
        if (VC) {
            const u64 *A = m.A(l);
            gc[J] = tau_rhs_vc(restrict_rhs(g[i0], g[i0 + 1]), um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, 2 * l - 4,
                               A[i0], A[i0 + 2]);
        } else {
            gc[J] = tau_rhs(restrict_rhs(g[i0], g[i0 + 1]), um2, um1, u[i0], u[i0 + 1], u2, u3, J, nc, 2 * l - 4);
        }
    }
    __syncthreads();
}

// The coarsest level of -(a u')' = f in FP64: Thomas on the level's operator
// with the FP64 face coefficients a (G 2^-(Sg0 + 2 M0) is h^2 rhs of -(a u')'
// = f: the normalisation 2^-Ea of the fixed-point levels is folded into Sg0),
// row i: -a_i u_{i-1} + (a_i + a_{i+1}) u_i - a_{i+1} u_{i+1} (a wall face
// counted twice), the result onto the fixed-point grid.  One thread.
__device__ void tail_coarsest_vc(TailSmem &m, const double *a, const Scale *sc) {
    const int n0 = 1 << m.M0;
    i64 *u = m.u + m.off(m.M0);
    const i64 *g = m.g + m.off(m.M0);
    if (threadIdx.x == 0) {
        const int gexp = sc->Sg0 + 2 * m.M0, S = sc->S;
        double *cp = reinterpret_cast<double *>(m.S), *dp = cp + n0;
        for (int i = 0; i < n0; ++i) {
            const double ai = a[i], ai1 = a[i + 1];
            const double al = (i == 0) ? scale2(ai, 1) : ai;
            const double ar = (i == n0 - 1) ? scale2(ai1, 1) : ai1;
            const double lower = (i > 0) ? -ai : 0.0, upper = (i < n0 - 1) ? -ai1 : 0.0;
            const double gi = fixed_to_f64(g[i], gexp);
            const double denom = (i > 0) ? (al + ar) - lower * cp[i - 1] : al + ar;
            cp[i] = upper / denom;
            dp[i] = ((i > 0) ? gi - lower * dp[i - 1] : gi) / denom;
        }
        double x = dp[n0 - 1];
        u[n0 - 1] = f64_to_fixed(x, S);
        for (int i = n0 - 2; i >= 0; --i) {
            x = dp[i] - cp[i] * x;
            u[i] = f64_to_fixed(x, S);
        }
    }
    __syncthreads();
}

// U_M0 = A^{-1} g in FP64: value u = A^{-1} (G 2^-(Sg0+2 M0)) times 2^S.
__device__ void tail_coarsest(TailSmem &m, const double *Ainv, const Scale *sc) {
    const int n0 = 1 << m.M0;
    i64 *u = m.u + m.off(m.M0);
    const i64 *g = m.g + m.off(m.M0);
    const int gexp = sc->Sg0 + 2 * m.M0, S = sc->S;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n0; ++j) s = fma(Ainv[i * n0 + j], fixed_to_f64(g[j], gexp), s);
        m.S[i] = f64_to_fixed(s, S);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) u[i] = m.S[i];
    __syncthreads();
}

template <bool VC>
__device__ void tail_up(TailSmem &m, int l, int nu) {
    const int n = 1 << l, nc = n >> 1;
    i64 *u = m.u + m.off(l);
    const i64 *uc = m.u + m.off(l - 1);
    for (int J = threadIdx.x; J < nc; J += blockDim.x) m.S[J] = uc[J] - ((u[2 * J] + u[2 * J + 1]) >> 1);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int J = i >> 1, nb = (i & 1) ? J + 1 : J - 1;
        i64 cn = (nb < 0) ? -m.S[0] : ((nb >= nc) ? -m.S[nc - 1] : m.S[nb]);
        u[i] += (3 * m.S[J] + cn + 2) >> 2;
    }
    __syncthreads();
    tail_smooth<VC>(m, l, nu);
}

__device__ void tail_interp(TailSmem &m, int l) {
    const int n = 1 << l, nc = n >> 1;
    const i64 *uc = m.u + m.off(l - 1);
    i64 *u = m.u + m.off(l);
    for (int j = (int)threadIdx.x - 2; j < nc + 2; j += (int)blockDim.x)
        if (j >= -2) m.S[j + 2] = coarse_reflect(uc, j, nc);
    __syncthreads();
    for (int J = threadIdx.x; J < nc; J += blockDim.x) fmg_interp2(m.S, -2, J, u[2 * J], u[2 * J + 1]);
    __syncthreads();
}

template <bool VC>
__global__ void __launch_bounds__(kTailBlock) tail_kernel(const __grid_constant__ TailArgs a) {
    pdl_enter();
    extern __shared__ i64 smi[];
    TailSmem m;
    m.M0 = a.M0;
    const int tot = (1 << (a.Mc + 1)) - (1 << a.M0);
    m.u = smi;
    m.g = m.u + tot;
    m.S = m.g + tot;
    m.X = m.S + (1 << a.Mc) + 8;
    m.Y = m.X + blockDim.x;
    m.cA = a.cA;
    m.cBM = a.cBM;
    const int nMc = 1 << a.Mc;
    const Scale *sc = a.sc + blockIdx.y;
    m.Kb = VC ? sc->Kb : 0;
    const double *coef0 = VC ? batch_at(a.coef0, (1LL << a.M0) + 1) : nullptr;
    auto coarsest = [&]() {
        if (VC) tail_coarsest_vc(m, coef0, sc);
        else tail_coarsest(m, a.Ainv, sc);
    };
    const i64 *u_in = batch_at(a.u_in, nMc), *g_in = batch_at(a.g_in, nMc);
    const double *f = batch_at(a.f, nMc);
    i64 *u_out = batch_at(a.u_out, nMc);
    double *u_out_f64 = batch_at(a.u_out_f64, nMc);
    const int kg = sc->Sg0;
    if (g_in) stage_range(m.g + m.off(a.Mc), g_in, nMc);
    else stage_range(m.g + m.off(a.Mc), f, nMc);
    if (a.mode == 1) stage_range(m.u + m.off(a.Mc), u_in, nMc);
    stage_wait();
    __syncthreads();
    if (!g_in)
        for (int i = threadIdx.x; i < nMc; i += blockDim.x)
            m.g[m.off(a.Mc) + i] = f64_to_fixed(__longlong_as_double(m.g[m.off(a.Mc) + i]), kg);
    __syncthreads();
    if (a.mode == 0) {
        for (int l = a.Mc; l > a.M0; --l) {
            const i64 *g = m.g + m.off(l);
            i64 *gc = m.g + m.off(l - 1);
            for (int J = threadIdx.x; J < (1 << (l - 1)); J += blockDim.x) gc[J] = (g[2 * J] + g[2 * J + 1] + 1) >> 1;
            __syncthreads();
        }
        coarsest();
        for (int k = a.M0; k < a.Mc; ++k) {
            tail_interp(m, k + 1);
            for (int l = k + 1; l > a.M0; --l) tail_down<VC>(m, l, a.nu1);
            coarsest();
            for (int l = a.M0 + 1; l <= k + 1; ++l) tail_up<VC>(m, l, a.nu2);
        }
    } else {
        for (int l = a.Mc; l > a.M0; --l) tail_down<VC>(m, l, a.nu1);
        coarsest();
        for (int l = a.M0 + 1; l <= a.Mc; ++l) tail_up<VC>(m, l, a.nu2);
    }
    if (u_out_f64) {
        const int S = sc->S;
        for (int i = threadIdx.x; i < nMc; i += blockDim.x) u_out_f64[i] = fixed_to_f64(m.u[m.off(a.Mc) + i], S);
    } else {
        for (int i = threadIdx.x; i < nMc; i += blockDim.x) u_out[i] = m.u[m.off(a.Mc) + i];
    }
}

}  // namespace fx
}  // namespace srfmg
