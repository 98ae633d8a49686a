// vbc_device.cuh -- device-side types and per-pair arithmetic of the VBC.
//
// Positions live on the device as fixed-point fractions of the box edge:
// a coordinate x is stored as x / L * 2^B, rounded, modulo 2^B, with
// B = 32 (FP32-split mode, int4 per particle) or B = 64 (FP64 mode, 32-byte
// record).  The difference of two such words, read as a signed integer, is
// the minimum-image separation in units of L / 2^B, so the periodic wrap
// costs nothing and the separation is exact before it is rounded to
// floating point once.
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

// Unevaluated sum hi + lo of two floats (see the two-float helpers below).
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
    // fixed-point radii (units (L/2^32)^2) and threshold for the exact counts
    unsigned long long rl2_fix, rh2_fix;
    f2x rl_s, w_s;                    // r_l / s and (r_h - r_l) / s as two floats
    long long fd_int;                 // floor(f - delta)
    long long fd_frac_fix;            // (f - delta - fd_int) * 2^31, rounded
};

// Device-side status words shared by all kernels of a system.
// Each flag has one writer kernel, and no kernel reads a flag that it writes,
// so every early exit is uniform within a kernel launch.
struct Status {
    int rebuild;        // 1: neighbour list must be rebuilt (k_force sets, k_count clears)
    int overflow;       // 1: a list exceeded the capacity at the last build (k_nlist)
    int frozen;         // 1: a non-finite position or velocity was produced (k_force)
    int crowded;        // 1: a cell held more than MAX_CELL particles (k_scan_apply)
    int nonfinite;      // unused padding kept for layout stability
    int max_nnb;        // longest list found at the last build (uncapped)
    int frozen_iter;    // loop iteration at which the freeze happened
    long long nnb_sum;  // sum of list lengths at the last build
    long long rebuilds; // builds so far
    long long in_window;// particles inside the switching window at the last count
    long long pairs;    // pairs with r < r_c at the last energy evaluation
    long long iter;     // loop iteration now running (advanced by k_gate)
    long long step_base;// noise counter of iteration 0 of the current call
    long long graph_rebuild_runs;  // rebuild bodies a graph conditional executed
};

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
    const float k = 1.0f / 8388608.0f;
    const float u0 = ((float)(x.x >> 9) + 0.5f) * k;
    const float u1 = ((float)(x.y >> 9) + 0.5f) * k;
    const float u2 = ((float)(x.z >> 9) + 0.5f) * k;
    const float u3 = ((float)(x.w >> 9) + 0.5f) * k;
    const float r0 = sqrtf(-2.0f * logf(u0));
    const float r1 = sqrtf(-2.0f * logf(u2));
    float s0, c0;
    sincospif(2.0f * u1, &s0, &c0);
    return make_float3(r0 * c0, r0 * s0, r1 * cospif(2.0f * u3));
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

// ---------------------------------------------------------------- position modes
struct ModeF32 {
    using pos_t = int4;
    using real = float;
    using real2 = float2;
    static constexpr bool fp64 = false;

    __device__ __forceinline__ static int3 idelta(const int4& a, const int4& b)
    {
        return make_int3(a.x - b.x, a.y - b.y, a.z - b.z);
    }
    // minimum-image separation a - b in length units
    __device__ __forceinline__ static void delta(const int4& a, const int4& b, const Geom& g,
                                                 float& dx, float& dy, float& dz)
    {
        const int3 d = idelta(a, b);
        dx = (float)d.x * g.s32;
        dy = (float)d.y * g.s32;
        dz = (float)d.z * g.s32;
    }
    __device__ __forceinline__ static void delta64(const int4& a, const int4& b, const Geom& g,
                                                   double& dx, double& dy, double& dz)
    {
        const int3 d = idelta(a, b);
        dx = (double)d.x * g.s32d[0];
        dy = (double)d.y * g.s32d[1];
        dz = (double)d.z * g.s32d[2];
    }
    __device__ __forceinline__ static uint32_t hi32(const int4& p, int a)
    {
        return (uint32_t)(a == 0 ? p.x : (a == 1 ? p.y : p.z));
    }
    // fixed-point word of an unwrapped coordinate: round(x 2^32 / L) mod 2^32
    // (rounding to nearest halves the quantisation error of a separation)
    __device__ __forceinline__ static int4 from_x(double x, double y, double z, const Geom& g)
    {
        return make_int4((int)(uint32_t)__double2ll_rn(x * g.inv32[0]),
                         (int)(uint32_t)__double2ll_rn(y * g.inv32[1]),
                         (int)(uint32_t)__double2ll_rn(z * g.inv32[2]), 0);
    }
};

struct ModeF64 {
    using pos_t = P64;
    using real = double;
    using real2 = double2;
    static constexpr bool fp64 = true;

    __device__ __forceinline__ static void delta64(const P64& a, const P64& b, const Geom& g,
                                                   double& dx, double& dy, double& dz)
    {
        dx = (double)(long long)(a.x - b.x) * g.s64[0];
        dy = (double)(long long)(a.y - b.y) * g.s64[1];
        dz = (double)(long long)(a.z - b.z) * g.s64[2];
    }
    __device__ __forceinline__ static void delta(const P64& a, const P64& b, const Geom& g,
                                                 double& dx, double& dy, double& dz)
    {
        delta64(a, b, g, dx, dy, dz);
    }
    __device__ __forceinline__ static uint32_t hi32(const P64& p, int a)
    {
        const unsigned long long v = (a == 0 ? p.x : (a == 1 ? p.y : p.z));
        return (uint32_t)(v >> 32);
    }
    __device__ __forceinline__ static unsigned long long word(double x, double inv32)
    {
        const double t = x * inv32;
        const double fl = floor(t);
        const unsigned long long hi = (unsigned long long)(uint32_t)__double2ll_rd(fl);
        const unsigned long long lo = (unsigned long long)__double2uint_rz((t - fl) * 4294967296.0);
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

// ---------------------------------------------------------------- two-float arithmetic
// Unevaluated sums hi + lo of two floats (error-free transformations of
// Dekker and Knuth), about 48 significant bits from the FP32 pipes; B300 runs
// FP64 at a small fraction of its FP32 rate, so the few operations that need
// more than FP32 on the per-step path use these instead.
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
// Exact two-float value of an unsigned integer below 2^62.
__device__ __forceinline__ f2x f2x_from_u64(unsigned long long v)
{
    const float hi = __ull2float_rn(v);
    const long long rest = (long long)v - (long long)__float2ull_rn(hi);
    return {hi, __ll2float_rn(rest)};
}

// omega(r; r_l, r_h) * 2^31, rounded to an integer, for a separation inside
// the counting window.  Inputs are exact integers in units of s = L / 2^32:
// r2 = r^2 / s^2 and D = (r^2 - r_l^2) / s^2; rl_s = r_l / s and w_s =
// (r_h - r_l) / s are two-float constants.  With
//   t = (r - r_l) / w = (r^2 - r_l^2) / ((r + r_l) w)
// the cancellation of r - r_l happens in exact integers, and every later
// step keeps about 48 bits, so the result is the rounded weight of the
// fixed-point separation.
__device__ __forceinline__ unsigned long long window_weight_fix31(unsigned long long r2,
                                                                  unsigned long long D, f2x rl_s, f2x w_s)
{
    const f2x R2 = f2x_from_u64(r2);
    const f2x Dd = f2x_from_u64(D);
    // r = sqrt(r2): FP32 root plus one correction from the exact residual
    const float rh = sqrtf(R2.hi);
    const f2x sq = two_prod(rh, rh);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(R2.hi, sq.hi), sq.lo), R2.lo);
    const f2x r = fast_two_sum(rh, __fdividef(res, __fmul_rn(2.0f, rh)));
    // den = (r + r_l) w, then t = D / den with one remainder correction
    const f2x den = f2x_mul(f2x_add(r, rl_s), w_s);
    const float t0 = __fdividef(Dd.hi, den.hi);
    const f2x p = two_prod(t0, den.hi);
    const float rem = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(Dd.hi, p.hi), p.lo), Dd.lo), __fmul_rn(t0, den.lo));
    const f2x t = fast_two_sum(t0, __fdividef(rem, den.hi));
    // omega = ((1 - t)(1 + t))^2
    f2x a = two_sum(1.0f, -t.hi);
    a.lo = __fsub_rn(a.lo, t.lo);
    f2x b = two_sum(1.0f, t.hi);
    b.lo = __fadd_rn(b.lo, t.lo);
    const f2x q = f2x_mul(a, b);
    const f2x w = f2x_mul(q, q);
    long long v = __float2ll_rn(__fmul_rn(w.hi, 2147483648.0f)) + __float2ll_rn(__fmul_rn(w.lo, 2147483648.0f));
    v = v < 0 ? 0 : (v > 2147483648LL ? 2147483648LL : v);
    return (unsigned long long)v;
}

// ---------------------------------------------------------------- pair functions (FP64)
// Used by the FP64 pass kernels and by the FP64 energy/virial kernel.
__device__ __forceinline__ double omega_d(double x, double x1, double x2)
{
    if (x <= x1) return 1.0;
    if (x >= x2) return 0.0;
    const double t = (x - x1) / (x2 - x1);
    const double q = 1.0 - t * t;
    return q * q;
}
__device__ __forceinline__ double domega_d(double x, double x1, double x2)
{
    if (x <= x1 || x >= x2) return 0.0;
    const double w = x2 - x1;
    const double t = (x - x1) / w;
    return -4.0 * t * (1.0 - t * t) / w;
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
    const double q = 1.0 - u * u;
    return -c.E_a * q * q;
}
__device__ __forceinline__ double dVa_d(double r, const Coef& c)
{
    if (r <= c.r_r || r >= c.r_a) return 0.0;
    const double u = (r - c.rm) / c.h;
    return 4.0 * c.E_a * u * (1.0 - u * u) / c.h;
}

// Work stops (until the host intervenes) once any of these is raised.
__device__ __forceinline__ bool halted(const Status* st)
{
    return (st->frozen | st->crowded | st->overflow) != 0;
}

}  // namespace vbc
