// blocks.cuh -- the per-item bodies of the factorization: a panel's
// diagonal block (Sec. III step 1), a 64-row chunk of its panel TRSM (step 2)
// and one tile of a supernodal update with its fused scatter (step 3,
// Sec. V-B).  Each is a device function over one CTA of 256 threads; the
// level-by-level kernels (factor.cu) and the persistent work-queue kernel of
// the upper levels (fqueue.cu) call the same bodies.  Global data that other
// CTAs of the same launch may have written is read through L2 (__ldcg),
// except the inverted diagonal blocks, each of which owns whole cache lines.
#pragma once

#include "kernels.cuh"
#include "operand.cuh"

#include <type_traits>

namespace spx {

// ---------------------------------------------------------------------------
// Pivot arithmetic in FP64 with short dependency chains.  IEEE FP64 division
// and square root expand into long chains of dependent FP64 instructions, and
// a dependent FP64 instruction costs tens of times its throughput slot on
// this part, so the column-by-column pivots would dominate the diagonal
// kernels.  Instead:
//  * a float seed is cut from the double's bits with integer operations (no
//    FP64 conversion), refined by the FP32 unit (rsqrtf / reciprocal) and
//    widened back the same way;
//  * reciprocal: Newton's method on 1/y - d, written with the error term
//    e = 1 - d y so that two steps need three dependent FP64 operations
//    (y1 = y0 + y0 e, e1 = e^2, y2 = y1 + y1 e1);
//  * square root and its reciprocal together: Goldschmidt's iteration
//    (g -> sqrt(d), h -> 1/(2 sqrt(d)); r = 1/2 - g h; g += g r; h += h r),
//    two iterations, five dependent FP64 operations.
// Each iteration squares the relative error: 2^-22 -> 2^-44 -> below FP64
// rounding.  Magnitudes outside the FP32 normal range fall back to IEEE.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool float_seed(double d, float *f)
{
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -125 || e > 126) return false;
    const unsigned fb = (unsigned)((b >> 32) & 0x80000000u) | ((unsigned)(e + 127) << 23) |
                        (unsigned)((b >> 29) & 0x7FFFFF);
    *f = __uint_as_float(fb);
    return true;
}

__device__ __forceinline__ double widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xFF) - 127;
    const long long b = ((long long)(u & 0x80000000u) << 32) | ((long long)(e + 1023) << 52) |
                        ((long long)(u & 0x7FFFFF) << 29);
    return __longlong_as_double(b);
}

__device__ __forceinline__ double rcp_newton(double d)
{
    float f;
    if (!float_seed(d, &f)) return 1.0 / d;
    const float yf = 1.0f / f;
    if (!(fabsf(yf) > 1e-37f && fabsf(yf) < 1e37f)) return 1.0 / d;
    const double y0 = widen(yf);
    const double e0 = fma(-d, y0, 1.0);
    const double y1 = fma(y0, e0, y0);
    const double e1 = e0 * e0;
    return fma(y1, e1, y1);
}

// sqrt(d) and 1/sqrt(d) for d > 0.
__device__ __forceinline__ void sqrt_rsqrt(double d, double *s, double *rs)
{
    float f;
    if (d <= 0.0 || !float_seed(d, &f)) {
        *s = sqrt(d);
        *rs = 1.0 / *s;
        return;
    }
    const double y = widen(rsqrtf(f));
    double g = d * y, h = 0.5 * y;
    double r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
    r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
    *s = g;
    *rs = 2.0 * h;
}

__device__ __forceinline__ float rcp_newton(float d) { return 1.0f / d; }

// 1/d for a pivot on the diagonal-block chain, three dependent FP64
// operations: the seed y0 is the approximate FP32 reciprocal (rcp.approx,
// relative error below 2^-23) of d's leading bits, cut with integer
// operations, so |1 - d y0| < 2^-22; one third-order Newton-Raphson step
// y = y0 (1 + e + e^2), e = 1 - d y0, leaves the error e^3 < 2^-66, below
// FP64 rounding.  Magnitudes outside [2^-125, 2^126) take IEEE division.
__device__ __forceinline__ double rcp_pivot(double d)
{
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -125 || e > 125) return 1.0 / d;
    const unsigned fb = (unsigned)((b >> 32) & 0x80000000u) | ((unsigned)(e + 127) << 23) |
                        (unsigned)((b >> 29) & 0x7FFFFF);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float(fb)));
    const double y0 = widen(yf);
    const double er = fma(-d, y0, 1.0);
    const double t = fma(er, er, er);
    return fma(y0, t, y0);
}

// FP64 <-> FP32 conversions with integer operations (the conversion
// instructions occupy the FP64 pipe): round to nearest even, with zeros and
// the FP32 normal range handled inline and anything else (subnormal,
// overflow, inf, NaN) through the conversion instruction.
__device__ __forceinline__ float narrow_rn(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    if (((hi & 0x7FFFFFFFu) | lo) == 0u) return __uint_as_float(sign);
    const int fe = (int)((hi >> 20) & 0x7FF) - 896;
    if (fe < 1 || fe > 254) return __double2float_rn(d);
    unsigned f = sign | ((unsigned)fe << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;   // the 29 dropped bits: round half to even
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}

__device__ __forceinline__ double widen_exact(float f)
{
    const unsigned u = __float_as_uint(f);
    if ((u << 1) == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 255u) return (double)f;
    return widen(f);
}

template <typename T> __device__ __forceinline__ T from_f64(double d) { return (T)d; }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return narrow_rn(d); }
template <typename T> __device__ __forceinline__ double to_f64(T v) { return (double)v; }
template <> __device__ __forceinline__ double to_f64<float>(float v) { return widen_exact(v); }

// d > 0 on the bit pattern (an integer compare instead of an FP64 one)
__device__ __forceinline__ bool pos_bits(long long db) { return db > 0 && db <= 0x7FF0000000000000LL; }

// D = A B + D on the FP64 tensor path (mma m8n8k4): A(r, k) at lane 4r + k,
// B(k, n) at lane 4n + k, D(r, 2q + {0, 1}) at lane 4r + q.  It shares the
// SM's FP64 datapath, so it is used only in phases where no FP64 chain runs
// beside it.
__device__ __forceinline__ void dmma_f64(double &d0, double &d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

constexpr int kDB = 8;
constexpr long kDiagSpin = 1l << 22;   // polls of the hand-off counter before a diagonal block gives up

__device__ __forceinline__ double shfl_d(double v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

// ---------------------------------------------------------------------------
// Diagonal block of width <= W (W = 16, 32, 64; the block is padded with the
// identity to W).  On this part a warp issues one FP64 instruction per ~64
// cycles and the SM as a whole one per ~19 (conversions included), so the
// FP64 work is counted in instructions:
//  * the factorization runs in LDL^T form in FP64 -- per column one
//    reciprocal of the pivot (three FP64 operations), the multipliers, and
//    the in-block updates, with no square root on the chain; warps 0 and 1
//    own each 8-column block panel in registers (rows kb .. kb+31 and the
//    rest of the block); warp 0 runs the pivot chain and hands each column's
//    reciprocal and block-row entries to warp 1 through shared memory (a
//    counter, bounded wait), the other warps apply the trailing updates; the
//    next block's columns are updated between the panels (on the FP64 tensor
//    path for W = 64, where nothing else runs);
//  * pivot tests and FP64 <-> FP32 conversions on the bit patterns;
//  * L = l diag(sqrt(d)) is formed afterwards, all columns in parallel;
//  * L^{-1} = diag(1/sqrt(d)) l^{-1}: FP32 factors invert the unit-lower l
//    by forward substitution in registers (warp v owns columns v, v + 8, ...);
//    FP64 factors by blocks (8 x 8 diagonal blocks by single lanes, then
//    pairs of blocks merged with X21 = -C^{-1} (B A^{-1})), which does a
//    sixth of the multiply-adds.
// ---------------------------------------------------------------------------
template <typename T, int W, bool ldlt>
__device__ __forceinline__ void ldl_diag_block(const DevPlan &p, int pid, T *__restrict__ L,
                                               T *__restrict__ Dinv, double replace_tau, int64_t *err_col,
                                               unsigned long long *nrepl, unsigned long long *nneg, double *sm)
{
    constexpr int LD = W + 1;
    constexpr int NT = 256;
    double *a = sm;                          // W x LD, FP64 working block
    double *lA = a + W * LD;                 // 2 x (W x kDB) unscaled block columns (ld W)
    double *dv = lA + 2 * W * kDB;           // pivots
    double *rsv = dv + W;                    // 1 / sqrt(pivot)
    double *hand = rsv + W;                  // per block-panel column: block rows' entries (8) and 1 / pivot
    volatile int *hflag = reinterpret_cast<volatile int *>(hand + 9 * kDB);   // columns handed to warp 1
    T *x = reinterpret_cast<T *>(hand + 9 * kDB + 8);   // W x LD inverse workspace
    T *tmp = x + W * LD;                     // (W/2)^2, the FP64 factors' inverse
    T *dvf = tmp + (W / 2) * (W / 2);        // pivots (Cholesky: their square roots) in T
    T *rvf = dvf + W;                        // and their reciprocals
    const int w = p.pw[pid], h = p.ph[pid];
    const int64_t col0 = p.pfcol[pid];
    T *D = L + p.pval[pid];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the block, padded with the identity to W: every load of a thread is
    // issued before its first store, so the loads overlap
    {
        constexpr int NPER = (W * W + NT - 1) / NT;
        T vv[NPER];
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int idx = tid + q * NT;
            const int i = idx % W, j = idx / W;
            vv[q] = (idx < W * W && i < w && j < w && i >= j) ? __ldcg(D + i + (int64_t)j * h) : (T)0;
        }
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
            const int idx = tid + q * NT;
            if (idx >= W * W) continue;
            const int i = idx % W, j = idx / W;
            a[i + j * LD] = (i < w && j < w) ? to_f64<T>(vv[q]) : (i == j ? 1.0 : 0.0);
        }
        if (tid == 0) *hflag = 0;
    }
    __syncthreads();

    // Block panel b by warp 0 (registers, two row sets of 32), writing the
    // multipliers into a and the unscaled block columns into lA (two buffers,
    // one per block parity, so that the next panel can overlap the trailing
    // update of the previous one).
    // Block panel kb (8 columns), rows in registers, by one warp per row set:
    //   role 0 (warp 0): rows kb .. kb+31, the pivots and their side effects;
    //   role 1 (warp 1, when rows kb+32.. exist): rows kb+32 .. kb+63.
    // Warp 1 recomputes the 8 x 8 diagonal part from its own copy of rows
    // kb .. kb+7 (lane l holds row kb + (l & 7)) with the same operations in
    // the same order as warp 0, so its pivots and multipliers are bit-equal
    // and the two warps never wait for each other.  Multipliers go to a, the
    // unscaled block columns to lA (two buffers, one per block parity, so
    // that the next panel can overlap the trailing update of the previous).
    const bool tau_pos = replace_tau > 0.0;
    const long long tau_bits = tau_pos ? __double_as_longlong(replace_tau) : 0;
    auto panel = [&](int kb, int role, bool two) {
        double *lAb = lA + ((kb / kDB) & 1) * (W * kDB);
        const int rq = kb + lane;                                 // role 0: rows of the pivot chain
        const int r1 = kb + 32 + lane;                            // role 1: its own rows
        double q[kDB], p1[kDB];
#pragma unroll
        for (int c = 0; c < kDB; ++c) {
            q[c] = (role == 0 && rq < W) ? a[rq + (kb + c) * LD] : 0.0;
            p1[c] = (role == 1 && r1 < W) ? a[r1 + (kb + c) * LD] : 0.0;
        }
        if (role == 1) {
            // the rows below: per column, the pivot's reciprocal and the block
            // rows' unscaled entries from warp 0 (bounded wait on its counter)
#pragma unroll
            for (int c = 0; c < kDB; ++c) {
                bool got = false;
                for (long it = 0; it < kDiagSpin; ++it)
                    if (*hflag >= kb + c + 1) {
                        got = true;
                        break;
                    }
                if (!got) {
                    if (lane == 0) atomicMin((long long *)err_col, -1ll);
                    break;
                }
                __threadfence_block();
                const double r = hand[c * 9 + 8];
                const double pl = p1[c] * r;
#pragma unroll
                for (int c2 = c + 1; c2 < kDB; ++c2) p1[c2] = fma(-pl, hand[c * 9 + c2], p1[c2]);
                if (r1 < W) lAb[r1 + c * W] = p1[c];
                p1[c] = pl;
            }
#pragma unroll
            for (int c = 0; c < kDB; ++c)
                if (r1 < W) a[r1 + (kb + c) * LD] = p1[c];
            return;
        }
#pragma unroll
        for (int c = 0; c < kDB; ++c) {
            const int k = kb + c;
            double d = shfl_d(q[c], c);                  // A(k, k) from lane c
            const bool report = role == 0 && lane == 0 && k < w;
            const long long db = __double_as_longlong(d);
            if constexpr (!ldlt) {                        // Cholesky: positive pivots
                if (!pos_bits(db)) {
                    if (report) {
                        if (tau_pos) atomicAdd(nrepl, 1ull);
                        else atomicMin((long long *)err_col, (long long)(col0 + k));
                    }
                    d = tau_pos ? replace_tau : 1.0;
                }
            } else {                                      // LDL^T: static pivoting
                const long long ab = db & 0x7FFFFFFFFFFFFFFFLL;   // |d| >= tau on the bits
                if (!(ab >= tau_bits && ab <= 0x7FF0000000000000LL) || (!tau_pos && ab == 0)) {
                    if (report) {
                        if (tau_pos) atomicAdd(nrepl, 1ull);
                        else atomicMin((long long *)err_col, (long long)(col0 + k));
                    }
                    d = tau_pos ? ((db < 0 && ab != 0 && ab <= 0x7FF0000000000000LL) ? -replace_tau : replace_tau)
                                : 1.0;
                }
                if (report && __double_as_longlong(d) < 0) atomicAdd(nneg, 1ull);
            }
            const double r = rcp_pivot(d);
            const double u0 = rq > k ? q[c] : 0.0;
            const double l0 = u0 * r;
            if (two) {   // hand the column to warp 1
                if (lane < kDB) hand[c * 9 + lane] = u0;
                if (lane == 0) hand[c * 9 + 8] = r;
                __syncwarp();
                __threadfence_block();
                if (lane == 0) *hflag = k + 1;
            }
#pragma unroll
            for (int c2 = c + 1; c2 < kDB; ++c2) {
                const double ac = shfl_d(u0, c2);                   // A(kb + c2, k)
                if (rq >= kb + c2) q[c2] = fma(-l0, ac, q[c2]);
            }
            if (rq < W) lAb[rq + c * W] = u0;
            q[c] = rq > k ? l0 : (rq == k ? 1.0 : 0.0);
            if (lane == c) dv[k] = d;
        }
#pragma unroll
        for (int c = 0; c < kDB; ++c)
            if (rq < W) a[rq + (kb + c) * LD] = q[c];
    };
    // Rank-kDB update by block kb of the lower part of columns [j0, j1),
    // rows >= j; the (i, j) pairs are spread densely over the threads
    // t0.. (stride ts) so that FP64 lanes are not wasted on the upper part.
    auto update = [&](int kb, int j0, int j1, int t0, int ts) {
        const double *lAb = lA + ((kb / kDB) & 1) * (W * kDB);
        // pairs ordered column by column: column j holds W - j rows
        int j = j0, rem = t0;      // pair e = t0, t0 + ts, ... decoded incrementally
        while (j < j1 && rem >= W - j) {
            rem -= W - j;
            ++j;
        }
        for (; j < j1;) {
            const int i = j + rem;
            // one accumulator from the entry itself: eight FP64 instructions
            // a pair, the fewest for the FP64 units the pivot chain shares
            double s = a[i + j * LD];
#pragma unroll
            for (int c = 0; c < kDB; ++c) s = fma(-a[i + (kb + c) * LD], lAb[j + c * W], s);
            a[i + j * LD] = s;
            rem += ts;
            while (j < j1 && rem >= W - j) {
                rem -= W - j;
                ++j;
            }
        }
    };

    if (warp == 0) panel(0, 0, 32 < W);
    else if (warp == 1 && 32 < W) panel(0, 1, true);
    __syncthreads();
    for (int kb = 0; kb < W; kb += kDB) {
        const int nb = kb + kDB;                 // next block
        if (nb < W) {
            // columns of the next block first: W = 64 on the FP64 tensor path,
            // one 8-row tile per warp with the block's 8 columns split in two
            // k halves on independent accumulators; narrower blocks by every
            // thread on the FP64 pipe (measured faster there)
            if constexpr (W == 64) {
                if (warp < (W - nb) / 8) {
                    const int i0 = nb + 8 * warp, r = lane >> 2, q4 = lane & 3;
                    const double *lAb = lA + ((kb / kDB) & 1) * (W * kDB);
                    double *c = a + (i0 + r) + (nb + 2 * q4) * LD;
                    double c0 = c[0], c1 = c[LD], e0 = 0.0, e1 = 0.0;
                    const double a0 = -a[(i0 + r) + (kb + q4) * LD], a1 = -a[(i0 + r) + (kb + 4 + q4) * LD];
                    const double b0 = lAb[(nb + r) + q4 * W], b1 = lAb[(nb + r) + (4 + q4) * W];
                    dmma_f64(c0, c1, a0, b0);
                    dmma_f64(e0, e1, a1, b1);
                    c[0] = c0 + e0;
                    c[LD] = c1 + e1;
                }
            } else {
                update(kb, nb, nb + kDB, tid, NT);
            }
            __syncthreads();
            // warps 0 (and 1) factor the next block while the others finish
            // this block's update
            const bool two = nb + 32 < W;
            if (warp == 0) panel(nb, 0, two);
            else if (warp == 1 && two) panel(nb, 1, true);
            else update(kb, nb + kDB, W, tid - (two ? 64 : 32), NT - (two ? 64 : 32));
            __syncthreads();
        }
    }

    // Cholesky: L = l diag(sqrt(d)), keep 1/sqrt(d) for the inverse.
    // LDL^T: store l (unit) with d on the diagonal, keep 1/d.
    if (tid < W) {
        if constexpr (ldlt) {
            rsv[tid] = rcp_newton(dv[tid]);
        } else {
            double sq, rs;
            sqrt_rsqrt(dv[tid], &sq, &rs);
            dv[tid] = sq;
            rsv[tid] = rs;
        }
        dvf[tid] = from_f64<T>(dv[tid]);
        rvf[tid] = from_f64<T>(rsv[tid]);
    }
    __syncthreads();
    for (int idx = tid; idx < W * W; idx += NT) {
        const int i = idx % W, j = idx / W;
        const T l = i > j ? from_f64<T>(a[i + j * LD]) : (T)0;
        if (i < w && j < w && i >= j)
            D[i + (int64_t)j * h] = i == j ? dvf[j] : (ldlt ? l : l * dvf[j]);
        x[i + j * LD] = i > j ? l : (i == j ? (T)1 : (T)0);
    }
    __syncthreads();

    T *Mi = Dinv + p.pinv[pid];
    if constexpr (std::is_same<T, float>::value) {
        // forward substitution in registers: warp v owns columns v, v + 8, ...
        // of X = l^{-1}, W / 32 rows per lane; at step k the lane holding row
        // k broadcasts x_k and every lane subtracts l(i, k) x_k.  The k loop
        // is split at the row-group boundary so that the broadcast reads a
        // fixed register.
        constexpr int CPW = W / 8;
        constexpr int RG = (W + 31) / 32;
        T xr[CPW][RG];
#pragma unroll
        for (int t = 0; t < CPW; ++t)
#pragma unroll
            for (int g = 0; g < RG; ++g) xr[t][g] = (32 * g + lane == warp + 8 * t) ? (T)1 : (T)0;
        auto step = [&](int k, auto gk) {
            constexpr int G = decltype(gk)::value;
            T lk[RG];
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                const int i = 32 * g + lane;
                const T v = x[min(i, W - 1) + k * LD];
                lk[g] = (i > k && i < W) ? v : (T)0;
            }
#pragma unroll
            for (int t = 0; t < CPW; ++t) {
                const T xk = __shfl_sync(0xffffffffu, xr[t][G], k & 31);
#pragma unroll
                for (int g = 0; g < RG; ++g) xr[t][g] = fmaf(-lk[g], xk, xr[t][g]);
            }
        };
        const int kmid = W < 32 ? W - 1 : 32;
        for (int k = warp; k < kmid; ++k) step(k, std::integral_constant<int, 0>());
        if constexpr (RG > 1)
            for (int k = 32; k < W - 1; ++k) step(k, std::integral_constant<int, RG - 1>());
        // Cholesky: L^{-1} = diag(1/sqrt(d)) l^{-1}.  LDL^T: l^{-1} below the
        // diagonal (unit), 1/d on it.
#pragma unroll
        for (int t = 0; t < CPW; ++t) {
            const int j = warp + 8 * t;
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                const int i = 32 * g + lane;
                if (i < w && j < w) {
                    T v;
                    if constexpr (ldlt) v = i > j ? xr[t][g] : (i == j ? rvf[i] : (T)0);
                    else v = i >= j ? xr[t][g] * rvf[i] : (T)0;
                    Mi[i + j * w] = v;
                }
            }
        }
    } else {
        // unit-lower inverse: 8 x 8 diagonal blocks first
        if (warp < W / kDB && lane < kDB) {
            const int o = warp * kDB, jj = lane;
            T xr[kDB];
#pragma unroll
            for (int q = 0; q < kDB; ++q) xr[q] = q == jj ? (T)1 : (T)0;
#pragma unroll
            for (int kk = 0; kk < kDB; ++kk) {
                if (kk >= jj) {
#pragma unroll
                    for (int ii = kk + 1; ii < kDB; ++ii) xr[ii] -= x[(o + ii) + (o + kk) * LD] * xr[kk];
                }
            }
            __syncwarp(0xffu);
#pragma unroll
            for (int ii = 0; ii < kDB; ++ii)
                if (ii > jj) x[(o + ii) + (o + jj) * LD] = xr[ii];
        }
        __syncthreads();
#pragma unroll
        for (int sz = kDB; sz < W; sz *= 2) {
            const int npair = W / (2 * sz);
            for (int e = tid; e < npair * sz * sz; e += NT) {
                const int pr = e / (sz * sz), rem = e % (sz * sz), i = rem % sz, j = rem / sz;
                const int o = pr * 2 * sz;
                T acc = (T)0;
                for (int k = j; k < sz; ++k) acc += x[(o + sz + i) + (o + k) * LD] * x[(o + k) + (o + j) * LD];
                tmp[pr * sz * sz + i + j * sz] = acc;
            }
            __syncthreads();
            for (int e = tid; e < npair * sz * sz; e += NT) {
                const int pr = e / (sz * sz), rem = e % (sz * sz), i = rem % sz, j = rem / sz;
                const int o = pr * 2 * sz;
                T acc = tmp[pr * sz * sz + i + j * sz];   // C^{-1} has a unit diagonal
                for (int k = 0; k < i; ++k) acc += x[(o + sz + i) + (o + sz + k) * LD] * tmp[pr * sz * sz + k + j * sz];
                x[(o + sz + i) + (o + j) * LD] = -acc;
            }
            __syncthreads();
        }
        // Cholesky: L^{-1} = diag(1/sqrt(d)) l^{-1}.  LDL^T: l^{-1} below the
        // diagonal (unit), 1/d on it.
        for (int idx = tid; idx < w * w; idx += NT) {
            const int i = idx % w, j = idx / w;
            if constexpr (ldlt) Mi[idx] = i > j ? x[i + j * LD] : (i == j ? rvf[i] : (T)0);
            else Mi[idx] = i >= j ? x[i + j * LD] * rvf[i] : (T)0;
        }
    }
}

template <typename T, int W>
__host__ __device__ constexpr size_t ldl_smem_bytes()
{
    return sizeof(double) * ((size_t)W * (W + 1) + (size_t)2 * W * kDB + 2 * W + 9 * kDB + 8) +
           sizeof(T) * ((size_t)W * (W + 1) + (size_t)(W / 2) * (W / 2) + 2 * (size_t)W);
}

// ---------------------------------------------------------------------------
// Panel TRSM (Sec. III step 2) as a product with the inverted diagonal block:
// rows [r0, r0+64) of the off-diagonal part X become X B with
//   LLT : B = L^{-T}           (B(k,j) = Linv(j,k))
//   LU_L: B = U^{-1}           (B(k,j) = Uinv(k,j))
//   LU_U: B = L^{-T}, unit L   (B(k,j) = Linv(j,k), 1 on the diagonal)
//   RIGHT_LINV: B = L^{-1}     (B(k,j) = Linv(k,j); the selected inversion's L_RJ L_JJ^{-1})
// The CTA copies its rows and the whole B operand of a 64-column tile to
// shared memory first (every load of a batch issued before its stores), so
// writing the rows back in place is safe and the K loop runs without
// barriers; 64 x 64 output tiles, 4 x 4 per thread, written back through
// shared memory in whole segments.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void trsm_chunk(const DevPlan &p, const RowChunk ch, const T *__restrict__ Dinv,
                                           T *__restrict__ X, int mode, void *opc, void *opc_lo, int kpad,
                                           int op_kind, T *__restrict__ Wout, unsigned char *smraw)
{
    constexpr int NB = 16;                     // loads in flight per thread while staging
    const int pid = ch.panel;
    const int w = p.pw[pid], h = p.ph[pid];
    const int wpad = (w + 15) & ~15;
    T *Xs = reinterpret_cast<T *>(smraw);      // Xs[k * 64 + r], k < wpad
    T *Bf = Xs + wpad * kTrsmRows;             // Bf[k * 65 + j], k < max(wpad, 64); then the output tile
    const T *Mi = Dinv + p.pinv[pid];
    T *Xg = X + p.pval[pid] + ch.r0;
    const int nr = min(kTrsmRows, h - ch.r0);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // B(k, j) of the product X B (see the table above).  Plain loads: every
    // panel's inverse starts on a 256-byte boundary and owns its cache lines,
    // and no CTA reads it before the panel's diagonal block has written it
    auto bval = [&](int k, int j) -> T {
        if (k >= w || j >= w) return (T)0;
        if (mode == TRSM_RIGHT_LINV) return k >= j ? Mi[k + j * w] : (T)0;
        if (mode == TRSM_LU_L) return k <= j ? Mi[k + j * w] : (T)0;
        if (j > k) return Mi[j + k * w];
        if (j == k) return (mode == TRSM_LU_U || mode == TRSM_LDLT) ? (T)1 : Mi[j + k * w];
        return (T)0;
    };
    // the chunk's rows, every load of a batch issued before its stores
    for (int base = tid; base < wpad * kTrsmRows; base += 256 * NB) {
        T v[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = base + 256 * q, r = e & 63, k = e >> 6;
            v[q] = (e < wpad * kTrsmRows && r < nr && k < w) ? __ldcg(Xg + r + (int64_t)k * h) : (T)0;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = base + 256 * q;
            if (e < wpad * kTrsmRows) Xs[e] = v[q];
        }
    }
    for (int c0 = 0; c0 < w; c0 += kUpdTile) {
        if (c0 > 0) __syncthreads();           // the previous tile is out of Bf
        for (int base = tid; base < wpad * kUpdTile; base += 256 * NB) {
            T v[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int e = base + 256 * q;
                v[q] = e < wpad * kUpdTile ? bval(e >> 6, c0 + (e & 63)) : (T)0;
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int e = base + 256 * q;
                if (e < wpad * kUpdTile) Bf[(e >> 6) * (kUpdTile + 1) + (e & 63)] = v[q];
            }
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
#pragma unroll 4
        for (int k = 0; k < wpad; ++k) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = Xs[k * 64 + tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bf[k * (kUpdTile + 1) + ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        if (mode == TRSM_LDLT) {
            // acc = X l^{-T} is the D L^T buffer row (Sec. V-B: the update then
            // multiplies L by it); L = acc D^{-1} goes back in place
            T *Wg = Wout + p.pval[pid] + ch.r0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = c0 + ty + 16 * b;
                const T dinv = j < w ? Mi[j + j * w] : (T)0;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int r = tx + 16 * a;
                    if (r >= nr || j >= w) continue;
                    Wg[r + (int64_t)j * h] = acc[a][b];
                    const T l = acc[a][b] * dinv;
                    Xg[r + (int64_t)j * h] = l;
                    if (opc)   // A operand: L; B operand: D L^T
                        put_operand(opc, opc_lo, (p.prow[pid] + ch.r0 + r) * kpad + j, op_kind, (float)l,
                                    (float)acc[a][b]);
                }
            }
            continue;
        }
        // the 64 x 64 result tile through shared memory, so that both the
        // column-major panel and the row-major operand copy are written in
        // whole segments
        __syncthreads();                       // every read of Bf is done
        T *Ot = Bf;                            // Ot[r * 65 + jj]
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Ot[(tx + 16 * a) * (kUpdTile + 1) + ty + 16 * b] = acc[a][b];
        __syncthreads();
        const int nc = min(kUpdTile, w - c0);
        for (int e = tid; e < nc * kTrsmRows; e += 256) {
            const int r = e & 63, jj = e >> 6;
            if (r < nr) Xg[r + (int64_t)(c0 + jj) * h] = Ot[r * (kUpdTile + 1) + jj];
        }
        if (opc) {
            // the same rows, K-major, for the tensor-core updates; columns
            // w .. c0+63 of the tile are zero and fill the row's padding
            const int64_t orow0 = p.prow[pid] + ch.r0;
            for (int e = tid; e < nr * kUpdTile; e += 256) {
                const int r = e >> 6, jj = e & 63;
                put_operand(opc, opc_lo, (orow0 + r) * kpad + c0 + jj, op_kind,
                            (float)Ot[r * (kUpdTile + 1) + jj], 0.0f);
            }
        }
    }
    if (opc) {
        // the rest of each operand row's padding
        const int64_t orow0 = p.prow[pid] + ch.r0;
        const int j0 = mode == TRSM_LDLT ? w : (w + kUpdTile - 1) / kUpdTile * kUpdTile;
        const int padw = kpad - j0;
        for (int e = tid; e < nr * padw; e += 256) {
            const int r = e / padw, j = j0 + e % padw;
            put_operand(opc, opc_lo, (orow0 + r) * kpad + j, op_kind, 0.0f, 0.0f);
        }
    }
}

template <typename T>
__host__ __device__ constexpr size_t trsm_smem_bytes(int wpad)
{
    return sizeof(T) * ((size_t)wpad * kTrsmRows + (size_t)(wpad > kUpdTile ? wpad : kUpdTile) * (kUpdTile + 1));
}

// ---------------------------------------------------------------------------
// Update with fused scatter (Sec. V-B).  One CTA computes a 64 x 64 tile of
// W = A_rows(M) * B_rows(N)^T over the source panel's width, K-chunked
// through shared memory, then subtracts it from the target panel at row
// relmap(i) and column row(j) - first column(target), with atomic adds so
// that sources of one level may hit the same target concurrently.
//   lower   : skip entries with i < j (Cholesky diagonal-block region)
//   from_r1 : rows below r1 only (the U^T side of an LU update)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void atomic_sub(T *addr, T v);
template <>
__device__ __forceinline__ void atomic_sub<double>(double *addr, double v) { atomicAdd(addr, -v); }
template <>
__device__ __forceinline__ void atomic_sub<float>(float *addr, float v) { atomicAdd(addr, -v); }

template <typename T, int TN>
__device__ __forceinline__ void update_tile(const DevPlan &p, const DevTask tk, const UpdTile tl,
                                            const T *__restrict__ Aop, const T *__restrict__ Bop,
                                            T *__restrict__ C, int lower, int from_r1, T *smem)
{
    // TM x TN output tile (64 x 64, or 256 x 16 for tasks facing few rows),
    // 4 x 4 outputs per thread, K-chunks of 16 staged in shared memory
    constexpr int TM = 4096 / TN;
    constexpr int RX = TM / 4, CX = TN / 4;      // thread grid: RX rows x 256/RX column groups
    T (*As)[TM + 1] = reinterpret_cast<T (*)[TM + 1]>(smem);
    T (*Bs)[TN + 1] = reinterpret_cast<T (*)[TN + 1]>(smem + 16 * (TM + 1));
    const int src = tk.src, tgt = tk.tgt;
    const int h = p.ph[src], K = p.pw[src];
    const int64_t sbase = p.pval[src];
    const T *A = Aop + sbase;
    const T *B = Bop + sbase;
    const int tid = threadIdx.x;
    const int tx = tid % RX, ty = tid / RX;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        if constexpr (TN == TM) {
            // loader: TM rows x 4 k per pass, A and B side by side
            const int lr = tid % TM, lk = tid / TM;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = lk + 4 * q;
                const int kg = k0 + kk;
                const int ra = tl.m0 + lr, rb = tl.n0 + lr;
                As[kk][lr] = (kg < K && ra < h) ? __ldcg(A + ra + (int64_t)kg * h) : (T)0;
                Bs[kk][lr] = (kg < K && rb < tk.r1) ? __ldcg(B + rb + (int64_t)kg * h) : (T)0;
            }
        } else {
            // loader: 256 rows x 1 k per pass for A, one 16 x 16 block for B
            static_assert(TM == 256 && TN == 16, "narrow tile is 256 x 16");
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int kg = k0 + kk, ra = tl.m0 + tid;
                As[kk][tid] = (kg < K && ra < h) ? __ldcg(A + ra + (int64_t)kg * h) : (T)0;
            }
            const int r = tid & 15, kk = tid >> 4;
            const int kg = k0 + kk, rb = tl.n0 + r;
            Bs[kk][r] = (kg < K && rb < tk.r1) ? __ldcg(B + rb + (int64_t)kg * h) : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + RX * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + CX * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
    const int hT = p.ph[tgt];
    T *Ct = C + p.pval[tgt];
    const int64_t fcolT = p.pfcol[tgt];
    const int32_t *srow = p.rows + p.prow[src];
    const int32_t *rmap = p.relmap + tk.relmap_off - tk.r0;
    const int rlo = from_r1 ? tk.r1 : tk.r0;
    int64_t coff[4];
    bool cok[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = tl.n0 + ty + CX * b;
        cok[b] = j < tk.r1;
        coff[b] = cok[b] ? (int64_t)(srow[j] - fcolT) * hT : 0;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = tl.m0 + tx + RX * a;
        if (i >= h || i < rlo) continue;
        const int64_t roff = rmap[i];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = tl.n0 + ty + CX * b;
            if (!cok[b] || (lower && i < j)) continue;
            atomic_sub<T>(Ct + roff + coff[b], acc[a][b]);
        }
    }
}

template <typename T, int TN>
__host__ __device__ constexpr size_t update_smem_elems()
{
    return (size_t)16 * (4096 / TN + 1) + (size_t)16 * (TN + 1);
}

}  // namespace spx
