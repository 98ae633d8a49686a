// vbc_kernels.cuh -- CUDA kernels of the VBC path (sm_103a).
//
// One step of the path, for N particles stored in Morton order of their cells:
//   rebuild (only when a particle moved more than skin/2 since the last build):
//     k_bin -> k_scan_sums -> k_scan_apply -> k_scatter -> k_cellsort ->
//     k_permute -> k_copyback -> k_nlist
//   k_count   pass 1: n_i, s_i, s'_i                        (Eqs. counter, Psidelta)
//   k_chain   A_i = s'_i sum_j s_j V_a(r_ij), window particles only
//   k_force   pass 2: F_i, fused with the BAOAB update of the state
//   k_energy  FP64 U, W and pair count (on request only)
// The rebuild kernels read a device flag and return at once when no rebuild
// is due, so the host never waits on the device between steps.  Every pass
// walks a full (both-direction) Verlet list, one thread per particle, and
// accumulates without atomics, so results do not depend on scheduling.
#pragma once

#include "vbc_device.cuh"

namespace vbc {

constexpr int TPB = 128;          // threads per block of the per-particle kernels
constexpr int SCAN_CHUNK = 2048;  // cells per block in the two-pass scan
constexpr int SCAN_TPB = 256;
constexpr int MAX_CELL = 512;     // a denser cell means the system has collapsed
constexpr int RED_TPB = 256;      // energy kernel block size

enum Epilogue { EPI_FORCE = 0, EPI_START = 1, EPI_FINISH = 2, EPI_FINISH_START = 3 };

// ================================================================ rebuild
template <class M>
__global__ void __launch_bounds__(TPB) k_bin(const typename M::pos_t* __restrict__ pos, int n,
                                             Geom g, const int* __restrict__ morton_rank,
                                             int* __restrict__ cell_of, int* __restrict__ slot_of,
                                             int* __restrict__ cell_count, Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        st->max_nnb = 0;
        st->nnb_sum = 0;
    }
    if (i >= n) return;
    const int3 c = cell_of_pos<M>(pos[i], g);
    const int key = morton_rank[(c.z * g.nc[1] + c.y) * g.nc[0] + c.x];
    cell_of[i] = key;
    slot_of[i] = atomicAdd(&cell_count[key], 1);
}

// Block-wide exclusive scan of one int per thread; returns the block total.
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) smem_warp[lane] = w;
    }
    __syncthreads();
    const int warp_off = warp > 0 ? smem_warp[warp - 1] : 0;
    total = smem_warp[NT / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

// Pass 1 of the scan: the sum of each chunk of SCAN_CHUNK cell counts.
__global__ void __launch_bounds__(SCAN_TPB) k_scan_sums(const int* __restrict__ cell_count, int ncell,
                                                        int* __restrict__ chunk_sum, const Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    __shared__ int sw[SCAN_TPB / 32];
    const int base = blockIdx.x * SCAN_CHUNK;
    int s = 0;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += SCAN_TPB) {
        const int c = base + k;
        if (c < ncell) s += cell_count[c];
    }
    int total;
    block_exclusive_scan<SCAN_TPB>(s, sw, total);
    if (threadIdx.x == 0) chunk_sum[blockIdx.x] = total;
}

// Pass 2: chunk offset from the preceding chunk sums, then the local scan.
// Writes cell_start[0..ncell] and clears cell_count for the next build.
__global__ void __launch_bounds__(SCAN_TPB) k_scan_apply(int* __restrict__ cell_count, int ncell,
                                                         const int* __restrict__ chunk_sum,
                                                         int* __restrict__ cell_start, Status* st)
{
    // raises `crowded` itself, so it does not test it
    if (!st->rebuild || st->frozen) return;
    __shared__ int sw[SCAN_TPB / 32];
    int off = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_TPB) off += chunk_sum[b];
    int tot;
    block_exclusive_scan<SCAN_TPB>(off, sw, tot);
    off = tot;  // sum over all preceding chunks
    constexpr int PER = SCAN_CHUNK / SCAN_TPB;
    const int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * PER;
    int v[PER];
    int s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = (base + k < ncell) ? cell_count[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = off + block_exclusive_scan<SCAN_TPB>(s, sw, total);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (base + k < ncell) {
            cell_start[base + k] = run;
            cell_count[base + k] = 0;
            if (v[k] > MAX_CELL) st->crowded = 1;
        }
        run += v[k];
    }
    if (base <= ncell - 1 && ncell - 1 < base + PER) cell_start[ncell] = run;
}

__global__ void __launch_bounds__(TPB) k_scatter(int n, const int* __restrict__ cell_of,
                                                 const int* __restrict__ slot_of,
                                                 const int* __restrict__ cell_start,
                                                 int* __restrict__ order, const Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    order[cell_start[cell_of[i]] + slot_of[i]] = i;
}

// Within each cell, order particles by their original index so that the
// layout (and every summation order) is independent of atomic scheduling.
__global__ void __launch_bounds__(TPB) k_cellsort(int ncell, const int* __restrict__ cell_start,
                                                  const int* __restrict__ id, int* __restrict__ order,
                                                  const Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int b = cell_start[c], e = cell_start[c + 1];
    for (int k = b + 1; k < e; ++k) {
        const int o = order[k];
        const int key = id[o];
        int m = k - 1;
        while (m >= b && id[order[m]] > key) {
            order[m + 1] = order[m];
            --m;
        }
        order[m + 1] = o;
    }
}

template <class M>
__global__ void __launch_bounds__(TPB) k_permute(int n, const int* __restrict__ order,
                                                 const double* __restrict__ x, const double* __restrict__ v,
                                                 const int* __restrict__ id,
                                                 const typename M::pos_t* __restrict__ pos,
                                                 double* __restrict__ xt, double* __restrict__ vt,
                                                 int* __restrict__ idt, typename M::pos_t* __restrict__ post,
                                                 const Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int o = order[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xt[(size_t)a * n + k] = x[(size_t)a * n + o];
        vt[(size_t)a * n + k] = v[(size_t)a * n + o];
    }
    idt[k] = id[o];
    post[k] = pos[o];
}

template <class M>
__global__ void __launch_bounds__(TPB) k_copyback(int n, const double* __restrict__ xt,
                                                  const double* __restrict__ vt, const int* __restrict__ idt,
                                                  const typename M::pos_t* __restrict__ post,
                                                  double* __restrict__ x, double* __restrict__ v,
                                                  int* __restrict__ id, typename M::pos_t* __restrict__ pos,
                                                  typename M::pos_t* __restrict__ xref, const Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[(size_t)a * n + k] = xt[(size_t)a * n + k];
        v[(size_t)a * n + k] = vt[(size_t)a * n + k];
    }
    id[k] = idt[k];
    const typename M::pos_t p = post[k];
    pos[k] = p;
    xref[k] = p;
}

// Squared separation compared against a squared radius: exact integers in the
// FP32 mode (cubic box), FP64 in the FP64 mode.
template <class M>
struct ListTest;
template <>
struct ListTest<ModeF32> {
    __device__ __forceinline__ static bool within(const int4& a, const int4& b, const Geom&,
                                                  unsigned long long r2fix, double)
    {
        const int dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                      (unsigned long long)((long long)dy * dy) +
                                      (unsigned long long)((long long)dz * dz);
        return r2 < r2fix;
    }
};
template <>
struct ListTest<ModeF64> {
    __device__ __forceinline__ static bool within(const P64& a, const P64& b, const Geom& g,
                                                  unsigned long long, double r2)
    {
        double dx, dy, dz;
        ModeF64::delta64(a, b, g, dx, dy, dz);
        return dx * dx + dy * dy + dz * dz < r2;
    }
};

// Verlet list of radius r_list: column-major nbr[k * n + i], k < cap.
template <class M>
__global__ void __launch_bounds__(TPB) k_nlist(int n, Geom g, const typename M::pos_t* __restrict__ pos,
                                               const int* __restrict__ morton_rank,
                                               const int* __restrict__ cell_start, unsigned long long rl2fix,
                                               double rl2, int cap, int* __restrict__ nbr,
                                               int* __restrict__ nnb, Status* st)
{
    // k_nlist raises `overflow` itself, so it does not test it
    if (!st->rebuild || st->frozen || st->crowded) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (i < n) {
        const typename M::pos_t pi = pos[i];
        const int3 c = cell_of_pos<M>(pi, g);
        for (int dz = -1; dz <= 1; ++dz) {
            int z = c.z + dz;
            z = z < 0 ? z + g.nc[2] : (z >= g.nc[2] ? z - g.nc[2] : z);
            for (int dy = -1; dy <= 1; ++dy) {
                int y = c.y + dy;
                y = y < 0 ? y + g.nc[1] : (y >= g.nc[1] ? y - g.nc[1] : y);
                for (int dx = -1; dx <= 1; ++dx) {
                    int x = c.x + dx;
                    x = x < 0 ? x + g.nc[0] : (x >= g.nc[0] ? x - g.nc[0] : x);
                    const int key = morton_rank[(z * g.nc[1] + y) * g.nc[0] + x];
                    const int b = cell_start[key], e = cell_start[key + 1];
                    for (int j = b; j < e; ++j) {
                        if (j == i) continue;
                        if (ListTest<M>::within(pi, pos[j], g, rl2fix, rl2)) {
                            if (cnt < cap) nbr[(size_t)cnt * n + i] = j;
                            ++cnt;
                        }
                    }
                }
            }
        }
        nnb[i] = cnt < cap ? cnt : cap;
        if (cnt > cap) {
            st->overflow = 1;
            st->frozen_iter = (int)st->iter;
        }
    }
    // block maximum and sum of the list lengths
    __shared__ int smax[TPB / 32];
    __shared__ long long ssum[TPB / 32];
    int m = cnt;
    long long s = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = m;
        ssum[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        m = smax[0];
        s = ssum[0];
        for (int w = 1; w < TPB / 32; ++w) {
            m = max(m, smax[w]);
            s += ssum[w];
        }
        atomicMax(&st->max_nnb, m);
        atomicAdd((unsigned long long*)&st->nnb_sum, (unsigned long long)s);
        if (blockIdx.x == 0) st->rebuilds += 1;
    }
}

// ================================================================ list walk
// Visits the list of particle i in batches of U entries: the U indices are
// loaded first (each a coalesced 128-byte row across the warp), then the U
// neighbour positions (gathers served by L1/L2), then the U pair bodies run.
// Batching keeps U independent loads in flight per thread, which the
// dependent index -> position chain would otherwise serialise.  Padding
// slots of the last batch point at i itself and are skipped.
template <class M, int U, class Body>
__device__ __forceinline__ void walk_list(int i, int n, int m, const int* __restrict__ nbr,
                                          const typename M::pos_t* __restrict__ pos, Body&& body)
{
    for (int k0 = 0; k0 < m; k0 += U) {
        int jj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jj[u] = (k0 + u < m) ? __ldg(nbr + (size_t)(k0 + u) * n + i) : i;
        typename M::pos_t pj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) pj[u] = pos[jj[u]];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u < m) body(jj[u], pj[u]);
    }
}

// ================================================================ pass 1: counts
// FP32-split: neighbours with r <= r_l add exactly 1 (an integer); window
// neighbours add omega in 2^-31 fixed point, evaluated from the exact integer
// r^2 - r_l^2.  The threshold test t = n - (f - delta) is taken in the same
// fixed point, so s_i and s'_i carry only the error of the window terms.
struct CountOut {
    double* n_out;          // counts in caller order, or null
    long long* in_window;   // counter of window particles, or null
};

__device__ __forceinline__ void switch_from_fix(long long T, float& s, float& ds)
{
    if (T <= 0) {
        s = 1.0f;
        ds = 0.0f;
    } else if (T >= 2147483648LL) {
        s = 0.0f;
        ds = 0.0f;
    } else {
        const float t = (float)T * 4.656612873077393e-10f;  // 2^-31
        const float q = 1.0f - t * t;
        s = q * q;
        ds = -4.0f * t * q;
    }
}

template <int U>
__global__ void __launch_bounds__(TPB) k_count_f32(int n, Geom g, Coef c, const int4* __restrict__ pos,
                                                   const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                   const int* __restrict__ id, float* __restrict__ ds_out,
                                                   float2* __restrict__ sA, CountOut out, Status* st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rebuild = 0;
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool win = false;
    if (i < n) {
        const int4 pi = pos[i];
        const int m = nnb[i];
        unsigned full = 0;
        unsigned long long q = 0;
        walk_list<ModeF32, U>(i, n, m, nbr, pos, [&](int, const int4& pj) {
            const int dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                          (unsigned long long)((long long)dy * dy) +
                                          (unsigned long long)((long long)dz * dz);
            if (r2 < c.rh2_fix) {
                if (r2 <= c.rl2_fix) {
                    ++full;
                } else {
                    q += window_weight_fix31(r2, r2 - c.rl2_fix, c.rl_s, c.w_s);
                }
            }
        });
        const long long T = ((long long)full - c.fd_int) * 2147483648LL + (long long)q - c.fd_frac_fix;
        float s, ds;
        switch_from_fix(T, s, ds);
        ds_out[i] = ds;
        sA[i] = make_float2(s, 0.0f);
        win = ds != 0.0f;
        if (out.n_out) out.n_out[id[i]] = (double)full + (double)q * 4.656612873077393e-10;
    }
    if (out.in_window) {
        const unsigned b = __ballot_sync(0xffffffffu, win);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd((unsigned long long*)out.in_window, (unsigned long long)__popc(b));
    }
}

__global__ void __launch_bounds__(TPB) k_count_f64(int n, Geom g, Coef c, const P64* __restrict__ pos,
                                                        const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                        const int* __restrict__ id, double* __restrict__ ds_out,
                                                        double2* __restrict__ sA, CountOut out, Status* st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rebuild = 0;
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool win = false;
    if (i < n) {
        const P64 pi = pos[i];
        const int m = nnb[i];
        double acc = 0.0;
        for (int k = 0; k < m; ++k) {
            const int j = nbr[(size_t)k * n + i];
            double dx, dy, dz;
            ModeF64::delta64(pi, pos[j], g, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
        }
        const double s = omega_d(acc, c.fd, c.fd + 1.0);
        const double ds = domega_d(acc, c.fd, c.fd + 1.0);
        ds_out[i] = ds;
        sA[i] = make_double2(s, 0.0);
        win = ds != 0.0;
        if (out.n_out) out.n_out[id[i]] = acc;
    }
    if (out.in_window) {
        const unsigned b = __ballot_sync(0xffffffffu, win);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd((unsigned long long*)out.in_window, (unsigned long long)__popc(b));
    }
}

// ================================================================ chain-rule pass
// A_i = s'_i sum_j s_j V_a(r_ij) for particles inside the switching window.
template <class M, int U>
__global__ void __launch_bounds__(TPB) k_chain(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                               const int* __restrict__ nbr, const int* __restrict__ nnb,
                                               const typename M::real* __restrict__ ds,
                                               typename M::real2* __restrict__ sA, const Status* st)
{
    using real = typename M::real;
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const real dsi = ds[i];
    if (dsi == (real)0) return;
    const typename M::pos_t pi = pos[i];
    const int m = nnb[i];
    const real* s_only = reinterpret_cast<const real*>(sA);  // s_j at even offsets
    real acc = 0;
    walk_list<M, U>(i, n, m, nbr, pos, [&](int j, const typename M::pos_t& pj) {
        real dx, dy, dz;
        M::delta(pi, pj, g, dx, dy, dz);
        const real r2 = dx * dx + dy * dy + dz * dz;
        if constexpr (M::fp64) {
            if (r2 > c.rr2 && r2 < c.ra2) acc += s_only[2 * j] * Va_d(sqrt(r2), c);
        } else {
            if (r2 > c.rr2f && r2 < c.ra2f) {
                const float r = sqrtf(r2);
                const float u = (r - c.rmf) * c.hinvf;
                const float q = 1.0f - u * u;
                acc += s_only[2 * j] * (-c.Eaf * q * q);
            }
        }
    });
    sA[i].y = dsi * acc;
}

// ================================================================ pass 2: forces + BAOAB
struct StepArgs {
    double* x;            // [3][n] unwrapped positions (FP64)
    double* v;            // [3][n] velocities (FP64)
    double* F_out;        // forces in caller order [n][3], or null (EPI_FORCE)
    double dt, c1, c2;    // BAOAB constants: c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT)
    unsigned long long seed;
    float half_skin2;     // (skin / 2)^2
};

template <class M, int EPI, int U>
__global__ void __launch_bounds__(TPB) k_force(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                               const int* __restrict__ nbr, const int* __restrict__ nnb,
                                               const int* __restrict__ id,
                                               const typename M::real2* __restrict__ sA,
                                               typename M::pos_t* __restrict__ pos_next,
                                               const typename M::pos_t* __restrict__ xref, StepArgs a,
                                               Status* st)
{
    using real = typename M::real;
    // k_force raises `frozen` itself; a thread that sees it raised by another
    // thread of the same launch stops early, which only happens on the error path
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const typename M::pos_t pi = pos[i];
    const typename M::real2 sai = sA[i];
    const int m = nnb[i];
    real fx = 0, fy = 0, fz = 0;
    walk_list<M, U>(i, n, m, nbr, pos, [&](int j, const typename M::pos_t& pj) {
        real dx, dy, dz;
        M::delta(pi, pj, g, dx, dy, dz);
        const real r2 = dx * dx + dy * dy + dz * dz;
        if constexpr (M::fp64) {
            if (r2 >= c.rc2) return;
            const typename M::real2 saj = sA[j];
            const double r = sqrt(r2);
            double gr = dVr_over_r_d(r2, c);
            if (r > 0.0) gr += (sai.x * saj.x * dVa_d(r, c) + (sai.y + saj.y) * domega_d(r, c.r_l, c.r_h)) / r;
            fx -= gr * dx;
            fy -= gr * dy;
            fz -= gr * dz;
        } else {
            if (r2 >= c.rc2f) return;
            const float2 saj = __ldg(sA + j);
            const float rinv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
            const float r = r2 * rinv;
            float gr = 0.0f;                                   // g / r
            if (r2 < c.rr2f) gr = c.Er4f * (r2 * c.rr2invf - 1.0f);
            float gt = 0.0f;                                   // g from the well and the counts
            if (r2 > c.rr2f && r2 < c.ra2f) {
                const float u = (r - c.rmf) * c.hinvf;
                gt = sai.x * saj.x * c.Ea4hf * u * (1.0f - u * u);
            }
            if (r2 > c.rl2f && r2 < c.rh2f) {
                const float t = (r - c.rlf) * c.winvf;
                gt -= (sai.y + saj.y) * 4.0f * t * (1.0f - t * t) * c.winvf;
            }
            gr += gt * rinv;
            fx -= gr * dx;
            fy -= gr * dy;
            fz -= gr * dz;
        }
    });
    if constexpr (EPI == EPI_FORCE) {
        if (a.F_out) {
            const int o = id[i];
            a.F_out[3 * (size_t)o + 0] = (double)fx;
            a.F_out[3 * (size_t)o + 1] = (double)fy;
            a.F_out[3 * (size_t)o + 2] = (double)fz;
        }
    } else {
        // BAOAB on the FP64 state (unit mass, h = dt / 2)
        const double h = 0.5 * a.dt;
        double xs[3], vs[3];
        const double f3[3] = {(double)fx, (double)fy, (double)fz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xs[d] = a.x[(size_t)d * n + i];
            vs[d] = a.v[(size_t)d * n + i];
        }
        if constexpr (EPI == EPI_FINISH || EPI == EPI_FINISH_START) {
#pragma unroll
            for (int d = 0; d < 3; ++d) vs[d] += h * f3[d];      // B: closes the previous step
        }
        if constexpr (EPI == EPI_START || EPI == EPI_FINISH_START) {
            double z[3];
            // noise counter of the step this iteration starts
            const unsigned long long nstep = (unsigned long long)(st->step_base + st->iter);
            if constexpr (M::fp64) {
                const double3 xi = langevin_normals_d(a.seed, nstep, (uint32_t)id[i]);
                z[0] = xi.x; z[1] = xi.y; z[2] = xi.z;
            } else {
                const float3 xi = langevin_normals(a.seed, nstep, (uint32_t)id[i]);
                z[0] = xi.x; z[1] = xi.y; z[2] = xi.z;
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                vs[d] += h * f3[d];                               // B
                xs[d] += h * vs[d];                               // A
                vs[d] = a.c1 * vs[d] + a.c2 * z[d];               // O
                xs[d] += h * vs[d];                               // A
            }
        }
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bad |= !isfinite(xs[d]) || !isfinite(vs[d]);
            a.x[(size_t)d * n + i] = xs[d];
            a.v[(size_t)d * n + i] = vs[d];
        }
        if constexpr (EPI == EPI_START || EPI == EPI_FINISH_START) {
            const typename M::pos_t pn = M::from_x(xs[0], xs[1], xs[2], g);
            pos_next[i] = pn;
            // displacement since the last build, on the top 32 bits of the words
            const typename M::pos_t pr = xref[i];
            float r2 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float u = (float)(int)(M::hi32(pn, d) - M::hi32(pr, d)) * (float)g.s32d[d];
                r2 += u * u;
            }
            if (r2 > a.half_skin2) st->rebuild = 1;
        }
        if (bad) {
            st->nonfinite = 1;
            st->frozen = 1;
        }
    }
}

// ================================================================ FP64 energy / virial
// Requested energies are held to 1e-9 relative, which needs the switching
// factors to FP64 accuracy: the counts, s, s' and A are recomputed here in
// FP64 from the exact fixed-point separations (these kernels run only when U
// or W is asked for, never inside the step loop).
template <class M>
__global__ void __launch_bounds__(TPB) k_count_e(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                 const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                 double2* __restrict__ sd, const Status* st)
{
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const typename M::pos_t pi = pos[i];
    const int m = nnb[i];
    double acc = 0.0;
    for (int k = 0; k < m; ++k) {
        double dx, dy, dz;
        M::delta64(pi, pos[nbr[(size_t)k * n + i]], g, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
    }
    sd[i] = make_double2(omega_d(acc, c.fd, c.fd + 1.0), domega_d(acc, c.fd, c.fd + 1.0));
}

template <class M>
__global__ void __launch_bounds__(TPB) k_chain_e(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                 const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                 const double2* __restrict__ sd, double* __restrict__ Ad,
                                                 const Status* st)
{
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dsi = sd[i].y;
    if (dsi == 0.0) {
        Ad[i] = 0.0;
        return;
    }
    const typename M::pos_t pi = pos[i];
    const int m = nnb[i];
    double acc = 0.0;
    for (int k = 0; k < m; ++k) {
        const int j = nbr[(size_t)k * n + i];
        double dx, dy, dz;
        M::delta64(pi, pos[j], g, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > c.rr2 && r2 < c.ra2) acc += sd[j].x * Va_d(sqrt(r2), c);
    }
    Ad[i] = dsi * acc;
}

// Per-block partial sums of U = sum_{i<j} [V_r + s_i s_j V_a], W = sum_{i<j} -g r and
// of the number of pairs with r < r_c, each pair seen from both ends (halves).
template <class M>
__global__ void __launch_bounds__(RED_TPB) k_energy(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                    const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                    const double2* __restrict__ sd, const double* __restrict__ Ad,
                                                    double* __restrict__ partial, long long* __restrict__ ppairs,
                                                    const Status* st)
{
    __shared__ double se[RED_TPB], sw[RED_TPB];
    __shared__ long long sp[RED_TPB];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, w = 0.0;
    long long pairs = 0;
    if (i < n && !halted(st)) {
        const typename M::pos_t pi = pos[i];
        const double si = sd[i].x, Ai = Ad[i];
        const int m = nnb[i];
        for (int k = 0; k < m; ++k) {
            const int j = nbr[(size_t)k * n + i];
            double dx, dy, dz;
            M::delta64(pi, pos[j], g, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= c.rc2) continue;
            ++pairs;
            const double sj = sd[j].x, Aj = Ad[j];
            const double r = sqrt(r2);
            e += 0.5 * (Vr_d(r2, c) + si * sj * Va_d(r, c));
            const double gg = dVr_over_r_d(r2, c) * r + si * sj * dVa_d(r, c) +
                              (Ai + Aj) * domega_d(r, c.r_l, c.r_h);
            w += 0.5 * (-gg * r);
        }
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    sp[threadIdx.x] = pairs;
    __syncthreads();
    for (int s = RED_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
            sp[threadIdx.x] += sp[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = se[0];
        partial[2 * blockIdx.x + 1] = sw[0];
        ppairs[blockIdx.x] = sp[0];
    }
}

// Fixed-order sum of the block partials: out[0] = U, out[1] = W; pairs / 2 -> Status.
__global__ void __launch_bounds__(RED_TPB) k_reduce_final(int nb, const double* __restrict__ partial,
                                                          const long long* __restrict__ ppairs,
                                                          double* __restrict__ out, Status* st)
{
    __shared__ double se[RED_TPB], sw[RED_TPB];
    __shared__ long long sp[RED_TPB];
    double e = 0.0, w = 0.0;
    long long p = 0;
    for (int b = threadIdx.x; b < nb; b += RED_TPB) {
        e += partial[2 * b];
        w += partial[2 * b + 1];
        p += ppairs[b];
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    sp[threadIdx.x] = p;
    __syncthreads();
    for (int s = RED_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
            sp[threadIdx.x] += sp[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = se[0];
        out[1] = sw[0];
        st->pairs = sp[0] / 2;
    }
}

// ================================================================ state I/O
// Caller order [n][3] -> internal SoA in sorted order, and fixed-point words.
template <class M>
__global__ void __launch_bounds__(TPB) k_load_state(int n, Geom g, const double* __restrict__ pos_in,
                                                    const double* __restrict__ vel_in, const int* __restrict__ id,
                                                    double* __restrict__ x, double* __restrict__ v,
                                                    typename M::pos_t* __restrict__ pos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
    double xs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d] = pos_in[3 * (size_t)o + d];
        x[(size_t)d * n + i] = xs[d];
        v[(size_t)d * n + i] = vel_in ? vel_in[3 * (size_t)o + d] : 0.0;
    }
    pos[i] = M::from_x(xs[0], xs[1], xs[2], g);
}

__global__ void __launch_bounds__(TPB) k_store_state(int n, const int* __restrict__ id, const double* __restrict__ x,
                                                     const double* __restrict__ v, double* __restrict__ pos_out,
                                                     double* __restrict__ vel_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (pos_out) pos_out[3 * (size_t)o + d] = x[(size_t)d * n + i];
        if (vel_out) vel_out[3 * (size_t)o + d] = v[(size_t)d * n + i];
    }
}

template <class M>
__global__ void __launch_bounds__(TPB) k_store_switch(int n, const int* __restrict__ id,
                                                      const typename M::real* __restrict__ ds,
                                                      const typename M::real2* __restrict__ sA,
                                                      double* __restrict__ s_out, double* __restrict__ ds_out,
                                                      double* __restrict__ A_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
    if (s_out) s_out[o] = (double)sA[i].x;
    if (ds_out) ds_out[o] = (double)ds[i];
    if (A_out) A_out[o] = (double)sA[i].y;
}

__global__ void __launch_bounds__(TPB) k_store_nlist(int n, int cap_out, const int* __restrict__ id,
                                                     const int* __restrict__ nbr, const int* __restrict__ nnb,
                                                     int* __restrict__ nnb_out, int* __restrict__ nbr_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
    const int m = nnb[i];
    if (nnb_out) nnb_out[o] = m;
    if (nbr_out) {
        const int mm = m < cap_out ? m : cap_out;
        for (int k = 0; k < mm; ++k) nbr_out[(size_t)o * cap_out + k] = id[nbr[(size_t)k * n + i]];
    }
}

// Opens one loop iteration: advances the device iteration counter (which
// keys the Langevin noise) and, inside a CUDA graph, sets the conditional
// that runs the rebuild body only when a rebuild is due.
__global__ void k_gate(Status* st, cudaGraphConditionalHandle h, int in_graph)
{
    st->iter += 1;
    if (in_graph) {
        const bool due = st->rebuild && !halted(st);
        if (due) st->graph_rebuild_runs += 1;
        cudaGraphSetConditional(h, due ? 1u : 0u);
    }
}

__global__ void k_set_iter(Status* st, long long iter, long long step_base)
{
    st->iter = iter;
    st->step_base = step_base;
}

__global__ void k_iota(int n, int* __restrict__ id)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = i;
}

}  // namespace vbc
