// vbc_device.cuh -- device-side types and per-pair arithmetic of the VBC.
//
// Positions live on the device in fixed point.  For the pair walks, a
// coordinate x is stored as x / L * 2^B, rounded, modulo 2^B, with B = 32
// (FP32-split mode, int4 per particle) or B = 64 (FP64 mode, 32-byte record).
// The difference of two such words, read as a signed integer, is the
// minimum-image separation in units of L / 2^B: the periodic wrap costs
// nothing and the separation is exact before it is rounded once.
//
// B300 executes FP64 arithmetic, and 64-bit integer <-> floating-point
// conversions, on a narrow pipe (a small fraction of the FP32 rate).  The
// per-step kernels of the FP32-split mode therefore contain no FP64
// instruction at all: exact integers carry what needs more than 24 bits, and
// the few quantities that need about 48 bits are two-float values
// (unevaluated sums hi + lo, Dekker/Knuth error-free transformations).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vbc {

struct __align__(16) P64 {
    unsigned long long x, y, z, w;
};

// Box geometry and cell grid, passed to kernels by value.
struct Geom {
    double L[3];
    double inv32[3];   // 2^32 / L
    double s32d[3];    // L / 2^32
    double s64[3];     // L / 2^64
    float s32;         // L / 2^32 (cubic box, FP32 mode)
    float s32sq;       // (L / 2^32)^2
    int nc[3];         // cells per axis (>= 3)
    int ncell;
};

// Unevaluated sum hi + lo of two floats.
struct f2x {
    float hi, lo;
};

// Pair parameters with derived constants (Eqs. softcore, omega, Psidelta).
struct Coef {
    // FP64 copies
    double r_r, r_a, r_l, r_h, E_r, E_a, f, delta;
    double rr2, ra2, rl2, rh2, rc2, rm, h, w, fd;
    // FP32 copies for the split mode
    float rr2f, ra2f, rl2f, rh2f, rc2f;
    float rlf, rmf, hinvf, winvf, wf;
    float Er4f;    // 4 E_r / r_r^2
    float rr2invf; // 1 / r_r^2
    float Eaf;     // E_a
    float Ea4hf;   // 4 E_a / h
    // exact fixed-point squared radii (units (L/2^32)^2) and the threshold for the counts
    unsigned long long rr2_fix, rl2_fix, rh2_fix, ra2_fix, rm2_fix, rc2_fix;
    float s2hinv;   // s^2 / h: u = (r^2 - r_m^2) / ((r + r_m) h) from an integer difference
    float s2winv;   // s^2 / w: t = (r^2 - r_l^2) / ((r + r_l) w)
    float rl2_fixf; // rl2_fix as a float (the chain-rule term of the FP32 force)
    f2x rl_s, w_s;                    // r_l / s and (r_h - r_l) / s as two floats, s = L / 2^32
    const uint4* wtab;                // window weights as cubic pieces in r^2 (window_weight_tab), or null
    int wsh;                          // log2 of the r^2 extent of one piece (fixed-point units)
    long long fd_int;                 // floor(f - delta)
    long long fd_frac_fix;            // (f - delta - fd_int) * 2^31, rounded
    long long fd_fix;                 // f - delta in 2^-31 fixed point: fd_int * 2^31 + fd_frac_fix (host-formed;
                                      // a count's threshold difference is n 2^31 + q - fd_fix)
    long long sat_full;               // ceil(f - delta + 1): this many neighbours inside r_l give s = s' = 0
};

// Device-side status words shared by all kernels of a system.
// Each flag has one writer kernel, and no kernel reads a flag that it writes,
// so every early exit is uniform within a kernel launch.
struct Status {
    int rebuild;        // 1: neighbour list must be rebuilt (k_step sets; k_count_rows, after both
                        // close counts, clears)
    int overflow;       // 1: a list exceeded the capacity at the last build (k_nlist)
    int frozen;         // 1: a non-finite position or velocity was produced (k_force)
    int crowded;        // 1: a cell held more than MAX_CELL particles (k_scan_apply)
    int max_stage;      // largest number of particles a supercell stages (last build)
    int max_nnb;        // longest list found at the last build (uncapped)
    int frozen_iter;    // loop iteration at which the overflow happened
    int max_own;        // largest number of particles of one supercell (last build)
    int stage_overflow; // 1: a supercell exceeded its staging or own-particle capacity (k_nlist)
    long long nnb_sum;  // sum of list lengths at the last build
    long long rebuilds; // builds so far
    long long in_window;// particles inside the switching window at the last count
    long long pairs;    // pairs with r < r_c at the last energy evaluation
    long long iter;     // loop iteration now running (advanced by k_gate)
    long long step_base;// noise counter of iteration 0 of the current call
    long long graph_rebuild_runs;  // rebuild bodies a graph conditional executed
    int nwin;           // window particles listed by the last count (k_count_rows)
    int nu;             // particles the last count walked in full: not saturated by their kept close
                        // neighbours (k_count_near)
    int ngen;           // particles whose force k_force_rows forms (k_count_near, k_chain)
    int bad_index;      // nonzero: a device-side index check failed (BadIndex; an internal error)
    int bad_input;      // 1: a loaded position or velocity was non-finite or beyond the fixed-point range (k_load_state)
    int aborted;        // 1: a batched iteration gave up waiting and left the state incomplete (host)
};

// Work stops (until the host intervenes) once any of these is raised.
__device__ __forceinline__ bool halted(const Status* st)
{
    return (st->frozen | st->crowded | st->overflow | st->stage_overflow | st->bad_input | st->aborted) != 0;
}

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of two 32x32
// multiplications with fixed multipliers, key advanced by Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Three standard normals for particle `pid` at step counter `step`: each word
// becomes u = ((x >> 9) + 1/2) / 2^23, exact in binary32, then Box-Muller.
__device__ __forceinline__ float3 langevin_normals(unsigned long long seed,
                                                   unsigned long long step, uint32_t pid)
{
    const uint4 x = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)(step >> 32), pid, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    // u = ((x >> 9) + 1/2) 2^-23, exactly, from the bits of 1 + (x >> 9) 2^-23
    const float half_ulp = 5.9604644775390625e-8f;  // 2^-24
    const float u0 = (__uint_as_float(0x3F800000u | (x.x >> 9)) - 1.0f) + half_ulp;
    const float u1 = (__uint_as_float(0x3F800000u | (x.y >> 9)) - 1.0f) + half_ulp;
    const float u2 = (__uint_as_float(0x3F800000u | (x.z >> 9)) - 1.0f) + half_ulp;
    const float u3 = (__uint_as_float(0x3F800000u | (x.w >> 9)) - 1.0f) + half_ulp;
    const float r0 = sqrtf(-2.0f * logf(u0));
    const float r1 = sqrtf(-2.0f * logf(u2));
    // angles 2 pi u taken as pi + 2 pi (u - 1/2): the hardware sine and cosine
    // are accurate to 2^-21.4 on [-pi, pi], and u - 1/2 is exact
    const float k2pi = 6.2831853071795864769f;
    float s0, c0;
    __sincosf(k2pi * (u1 - 0.5f), &s0, &c0);
    const float c3 = __cosf(k2pi * (u3 - 0.5f));
    return make_float3(-r0 * c0, -r0 * s0, -r1 * c3);
}

// Fixed-point product: nearest integer of v (hi + lo 2^-64), for |v| < 2^62
// and a non-negative factor with integer part hi and fraction lo 2^-64.
__device__ __forceinline__ long long mul_fix(long long v, unsigned long long hi, unsigned long long lo)
{
    const unsigned long long av = (unsigned long long)(v < 0 ? -v : v);
    const unsigned long long frac_lo = av * lo;
    unsigned long long r = av * hi + __umul64hi(av, lo) + (frac_lo >> 63);
    return v < 0 ? -(long long)r : (long long)r;
}

// The same three normals with the Box-Muller transform in FP64 (FP64 mode).
__device__ __forceinline__ double3 langevin_normals_d(unsigned long long seed,
                                                      unsigned long long step, uint32_t pid)
{
    const uint4 x = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)(step >> 32), pid, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double k = 1.0 / 8388608.0;
    const double u0 = ((double)(x.x >> 9) + 0.5) * k;
    const double u1 = ((double)(x.y >> 9) + 0.5) * k;
    const double u2 = ((double)(x.z >> 9) + 0.5) * k;
    const double u3 = ((double)(x.w >> 9) + 0.5) * k;
    const double r0 = sqrt(-2.0 * log(u0));
    const double r1 = sqrt(-2.0 * log(u2));
    double s0, c0;
    sincospi(2.0 * u1, &s0, &c0);
    return make_double3(r0 * c0, r0 * s0, r1 * cospi(2.0 * u3));
}

// ---------------------------------------------------------------- conversions on the ALU pipes
// Exact float of an unsigned integer below 2^23 (magic-number trick).
__device__ __forceinline__ float u23_to_float(uint32_t v)
{
    return __uint_as_float(0x4B000000u | v) - 8388608.0f;
}
// Nearest integer of a float with |x| < 2^62, as a 64-bit integer, from its bits.
__device__ __forceinline__ long long float_to_ll_rn(float x)
{
    const uint32_t u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xffu) - 150;  // |x| = m 2^e
    const unsigned long long m = (unsigned long long)((u & 0x7fffffu) | 0x800000u);
    unsigned long long v;
    if (e >= 0) {
        v = m << e;
    } else if (e > -25) {
        v = (m + (1ull << (-e - 1))) >> (-e);  // round half away from zero
    } else {
        v = 0ull;
    }
    return (u >> 31) ? -(long long)v : (long long)v;
}

// ---------------------------------------------------------------- two-float arithmetic
__device__ __forceinline__ f2x two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ f2x fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2x two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ f2x f2x_add(f2x a, f2x b)
{
    f2x s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ f2x f2x_mul(f2x a, f2x b)
{
    f2x p = two_prod(a.hi, b.hi);
    const float c = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return fast_two_sum(p.hi, __fadd_rn(p.lo, c));
}
// two-float times float
__device__ __forceinline__ f2x f2x_mulf(f2x a, float b)
{
    f2x p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// Nearest 64-bit integer of a two-float value (|value| < 2^62).
__device__ __forceinline__ long long f2x_to_ll(f2x a)
{
    const long long ih = float_to_ll_rn(a.hi);
    // a.hi - ih is exact: zero when |a.hi| >= 2^24 (a.hi is then an integer),
    // and |ih| < 2^24 is exactly a float otherwise
    const float base = fabsf(a.hi) < 16777216.0f ? __int2float_rn((int)ih) : a.hi;
    const float fr = __fadd_rn(__fsub_rn(a.hi, base), a.lo);
    return ih + float_to_ll_rn(fr);
}
// Float of an unsigned integer below 2^63 (within one unit in the last place),
// with only ALU/FMA operations.
__device__ __forceinline__ float u64_to_float(unsigned long long v)
{
    const float c2 = u23_to_float((uint32_t)(v >> 42)) * 4398046511104.0f;               // * 2^42
    const float c1 = u23_to_float((uint32_t)(v >> 21) & 0x1fffffu) * 2097152.0f;          // * 2^21
    const float c0 = u23_to_float((uint32_t)v & 0x1fffffu);
    return __fadd_rn(__fadd_rn(c2, c1), c0);
}
__device__ __forceinline__ float s64_to_float(long long v)
{
    const float f = u64_to_float((unsigned long long)(v < 0 ? -v : v));
    return v < 0 ? -f : f;
}

// Two-float value of an unsigned integer below 2^63, with only ALU/FMA operations:
// three exact 21-bit chunks summed with one error-free addition.
__device__ __forceinline__ f2x u64_to_f2x(unsigned long long v)
{
    const float c2 = u23_to_float((uint32_t)(v >> 42)) * 4398046511104.0f;               // * 2^42
    const float c1 = u23_to_float((uint32_t)(v >> 21) & 0x1fffffu) * 2097152.0f;          // * 2^21
    const float c0 = u23_to_float((uint32_t)v & 0x1fffffu);
    const f2x s = two_sum(c2, c1);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, c0));
}

// omega(r; r_l, r_h) * 2^31, rounded to an integer, for a separation inside
// the counting window.  Inputs are exact integers in units of s = L / 2^32:
// r2 = r^2 / s^2 and D = (r^2 - r_l^2) / s^2; rl_s = r_l / s and w_s =
// (r_h - r_l) / s are two-float constants.  With
//   t = (r - r_l) / w = (r^2 - r_l^2) / ((r + r_l) w)
// the cancellation in r - r_l happens in exact integers; r, r + r_l, the
// denominator and t carry two-float residuals (about 7e-9 RMS error in
// omega), and omega = ((1 - t)(1 + t))^2 is formed in 31-bit fixed point.
// No FP64 instruction and no 64-bit conversion is involved.
__device__ __forceinline__ unsigned long long window_weight_fix31(unsigned long long r2,
                                                                  unsigned long long D, f2x rl_s, f2x w_s)
{
    const f2x Dd = u64_to_f2x(D);
    const f2x R2 = u64_to_f2x(r2);
    // r = sqrt(r2), corrected once from the residual r2 - r^2
    const float rh = sqrtf(R2.hi);
    const float res = __fadd_rn(__fmaf_rn(-rh, rh, R2.hi), R2.lo);
    const float rlo = __fdividef(res, __fmul_rn(2.0f, rh));
    // a = r + r_l and den = a w as two floats
    f2x a = two_sum(rh, rl_s.hi);
    a = fast_two_sum(a.hi, __fadd_rn(a.lo, __fadd_rn(rl_s.lo, rlo)));
    const float dh = __fmul_rn(a.hi, w_s.hi);
    const float dl = __fadd_rn(__fmaf_rn(a.hi, w_s.hi, -dh), __fmaf_rn(a.hi, w_s.lo, __fmul_rn(a.lo, w_s.hi)));
    // t = D / den: leading quotient and the quotient of the exact remainder
    const float rcp = __frcp_rn(dh);
    const float th = __fmul_rn(Dd.hi, rcp);
    const float e = __fsub_rn(__fadd_rn(__fmaf_rn(-th, dh, Dd.hi), Dd.lo), __fmul_rn(th, dl));
    const float tl = __fmul_rn(e, rcp);
    long long t31 = float_to_ll_rn(__fmul_rn(th, 2147483648.0f)) + float_to_ll_rn(__fmul_rn(tl, 2147483648.0f));
    t31 = t31 < 0 ? 0 : (t31 > 2147483647LL ? 2147483647LL : t31);
    const unsigned long long q =
        ((2147483648ull - (unsigned long long)t31) * (2147483648ull + (unsigned long long)t31)) >> 31;
    return (q * q) >> 31;
}

// The same weight from a table of cubic pieces in r^2, for the list walks of
// the FP32-split counts.  Piece k covers D = r^2 - r_l^2 in [k 2^sh,
// (k + 1) 2^sh) (fixed-point units, exact integers); its entry holds omega at
// the piece's start in 2^-31 fixed point and the float coefficients of its
// cubic Hermite interpolant in the local coordinate u in [0, 1):
// omega = c0 + u (c1 + u (c2 + u c3)).  With 1024 pieces over the window the
// interpolation error is ~1e-13; the float part is at most the change of
// omega over one piece (~1e-3), so its rounding adds ~1e-10, and u keeps 23
// bits.  About 15 instructions against ~55 for window_weight_fix31.
__device__ __forceinline__ unsigned long long window_weight_tab(unsigned long long D, const uint4* __restrict__ tab,
                                                                int sh)
{
    const uint4 e = __ldg(tab + (int)(D >> sh));
    const unsigned long long low = D & ((1ull << sh) - 1ull);
    const uint32_t m = sh >= 23 ? (uint32_t)(low >> (sh - 23)) : (uint32_t)(low << (23 - sh));
    const float u = u23_to_float(m) * 1.1920928955078125e-7f;  // 2^-23
    const float d = u * __fmaf_rn(u, __fmaf_rn(u, __uint_as_float(e.w), __uint_as_float(e.z)), __uint_as_float(e.y));
    // |d| 2^31 < 2^22 (the change of omega over one piece), so a 32-bit conversion holds it
    const long long q = (long long)e.x + (long long)__float2int_rn(d * 2147483648.0f);
    return (unsigned long long)(q < 0 ? 0 : q);
}

// ---------------------------------------------------------------- position modes
struct ModeF32 {
    using pos_t = int4;
    using real = float;
    using real2 = float2;
    using xstate_t = long long;  // unwrapped position, fixed point in units of L / 2^52
    using vstate_t = long long;  // velocity, fixed point in units of 2^-40
    static constexpr bool fp64 = false;

    // minimum-image separation a - b in length units
    __device__ __forceinline__ static void delta64(const int4& a, const int4& b, const Geom& g,
                                                   double& dx, double& dy, double& dz)
    {
        dx = (double)(a.x - b.x) * g.s32d[0];
        dy = (double)(a.y - b.y) * g.s32d[1];
        dz = (double)(a.z - b.z) * g.s32d[2];
    }
    __device__ __forceinline__ static uint32_t hi32(const int4& p, int a)
    {
        return (uint32_t)(a == 0 ? p.x : (a == 1 ? p.y : p.z));
    }
    // 32-bit word of an unwrapped fixed-point coordinate P (units L / 2^52): round(P / 2^20) mod 2^32
    __device__ __forceinline__ static int word(long long P)
    {
        return (int)(uint32_t)((unsigned long long)(P + (1ll << 19)) >> 20);
    }
};

struct ModeF64 {
    using pos_t = P64;
    using real = double;
    using real2 = double2;
    using xstate_t = double;     // unwrapped position
    using vstate_t = double;     // velocity
    static constexpr bool fp64 = true;

    __device__ __forceinline__ static void delta64(const P64& a, const P64& b, const Geom& g,
                                                   double& dx, double& dy, double& dz)
    {
        dx = (double)(long long)(a.x - b.x) * g.s64[0];
        dy = (double)(long long)(a.y - b.y) * g.s64[1];
        dz = (double)(long long)(a.z - b.z) * g.s64[2];
    }
    __device__ __forceinline__ static uint32_t hi32(const P64& p, int a)
    {
        const unsigned long long v = (a == 0 ? p.x : (a == 1 ? p.y : p.z));
        return (uint32_t)(v >> 32);
    }
    __device__ __forceinline__ static unsigned long long word(double x, double inv32)
    {
        const double t = __dmul_rn(x, inv32);
        const double fl = floor(t);
        const unsigned long long hi = (unsigned long long)(uint32_t)__double2ll_rd(fl);
        const unsigned long long lo = (unsigned long long)__double2uint_rz(__dmul_rn(t - fl, 4294967296.0));
        return (hi << 32) | lo;
    }
    __device__ __forceinline__ static P64 from_x(double x, double y, double z, const Geom& g)
    {
        P64 p;
        p.x = word(x, g.inv32[0]);
        p.y = word(y, g.inv32[1]);
        p.z = word(z, g.inv32[2]);
        p.w = 0ull;
        return p;
    }
};

// Cell of a fixed-point position: c_a = floor(u_a nc_a / 2^32), always in [0, nc_a).
template <class M>
__device__ __forceinline__ int3 cell_of_pos(const typename M::pos_t& p, const Geom& g)
{
    return make_int3((int)(((unsigned long long)M::hi32(p, 0) * (unsigned)g.nc[0]) >> 32),
                     (int)(((unsigned long long)M::hi32(p, 1) * (unsigned)g.nc[1]) >> 32),
                     (int)(((unsigned long long)M::hi32(p, 2) * (unsigned)g.nc[2]) >> 32));
}

// ---------------------------------------------------------------- pair functions (FP64)
// Used by the FP64 mode and by the FP64 energy/virial evaluation.  Every
// product that feeds a sum is written as an explicit fused multiply-add (or an
// explicit product), so that the rounding of each result is fixed by the
// source and not by how the compiler contracts it in one kernel or another:
// the batched launch and the single-system kernels then agree bit for bit.
__device__ __forceinline__ double omega_d(double x, double x1, double x2)
{
    if (x <= x1) return 1.0;
    if (x >= x2) return 0.0;
    const double t = (x - x1) / (x2 - x1);
    const double q = __fma_rn(-t, t, 1.0);
    return __dmul_rn(q, q);
}
__device__ __forceinline__ double domega_d(double x, double x1, double x2)
{
    if (x <= x1 || x >= x2) return 0.0;
    const double w = x2 - x1;
    const double t = (x - x1) / w;
    return __dmul_rn(__dmul_rn(-4.0, t), __fma_rn(-t, t, 1.0)) / w;
}
__device__ __forceinline__ double Vr_d(double r2, const Coef& c)
{
    if (r2 >= c.rr2) return 0.0;
    const double q = 1.0 - r2 / c.rr2;
    return c.E_r * q * q;
}
// dV_r/dr divided by r (finite at r = 0)
__device__ __forceinline__ double dVr_over_r_d(double r2, const Coef& c)
{
    if (r2 >= c.rr2) return 0.0;
    return -4.0 * c.E_r / c.rr2 * (1.0 - r2 / c.rr2);
}
__device__ __forceinline__ double Va_d(double r, const Coef& c)
{
    if (r <= c.r_r || r >= c.r_a) return 0.0;
    const double u = (r - c.rm) / c.h;
    const double q = __fma_rn(-u, u, 1.0);
    return __dmul_rn(__dmul_rn(-c.E_a, q), q);
}
__device__ __forceinline__ double dVa_d(double r, const Coef& c)
{
    if (r <= c.r_r || r >= c.r_a) return 0.0;
    const double u = (r - c.rm) / c.h;
    return __dmul_rn(__dmul_rn(4.0 * c.E_a, u), __fma_rn(-u, u, 1.0)) / c.h;
}

}  // namespace vbc
