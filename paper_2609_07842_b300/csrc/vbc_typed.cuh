// vbc_typed.cuh -- several particle types with a count mask, and harmonic
// bonds (FP64 mode).
//
// The counter of a particle may run over chosen neighbour types only (Sec. 2),
// and the sticker model of Sec. 4 joins beads into bead-spring chains.  A
// typed system keeps the single-type machinery -- sorted order, cell groups,
// list rows of staging indices, the BAOAB update -- and replaces the three
// pair passes by the walks below, which take every pair's parameters from a
// table indexed by the two types:
//   n_i  = sum_{j: mask[t_i][t_j]} omega(r_ij; r_l^{ij}, r_h^{ij})
//   s_i  = omega(n_i; f_i - delta_i, f_i - delta_i + 1)   (f, delta of i's own type)
//   A_i  = s'_i sum_j s_j V_a^{ij}(r_ij)
//   g_ij = V_r^{ij}' + s_i s_j V_a^{ij}' + (mask[t_i][t_j] A_i + mask[t_j][t_i] A_j) omega^{ij}'
// and a bond (i, j) adds k_b (r - r_0) to g_ij; bonded pairs keep their
// non-bonded terms.  One warp per particle, one lane per list entry.  The
// FP64 mode uses FP64 pair arithmetic on the 64-bit fixed-point positions;
// the FP32-split mode (k_tcount32, k_tchain32, k_tforce32) the single-type
// split: exact integer squared separations of the 32-bit fixed-point words,
// integer counts plus 2^-31 fixed-point window weights (window pairs measured
// finer with the state's residual bits), FP32 pair and bond terms.  Energies
// and the virial are FP64 in both modes (k_tcount_e, k_tchain_e, k_tenergy).
#pragma once

#include "vbc_kernels.cuh"

namespace vbc {

constexpr int MAX_TYPES = 8;

struct TypedDev {
    const Coef* pc;         // [T * T] pair coefficients, row = type of i
    const int* mask;        // [T * T] 1: a particle of the row type counts neighbours of the column type
    int T;
    const int* type_orig;   // [n] type by original index
    int* tsort;             // [n] type by sorted index (refreshed after each list build)
    int* inv;               // [n] sorted index of each original index (idem)
    const long long* bptr;  // [n + 1] bond partners of original index o: bto[bptr[o] .. bptr[o + 1])
    const int* bto;         // partner original indices (each bond listed from both ends)
    double kb, r0;          // harmonic bond constant and rest length
};

// Types and inverse permutation in sorted order.  It depends on the order
// alone, so it may run whether or not a build took place.
__global__ void __launch_bounds__(TPB) k_tmaps(int n, const int* __restrict__ id, TypedDev t)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int o = id[p];
    t.tsort[p] = t.type_orig[o];
    t.inv[o] = p;
}

// Calls visit(j) for this lane's entries of particle p's row (j a sorted index).
template <class Visit>
__device__ __forceinline__ void typed_row(int p, const GroupAux& aux, const SuperCaps& cp,
                                          const uint16_t* __restrict__ nbr, const int* __restrict__ nnb,
                                          Visit&& visit)
{
    const int b = __ldg(aux.grp + p);
    const int* sidx = aux.stage_idx + (size_t)b * cp.smax;
    const uint16_t* row = nbr + (size_t)p * cp.cap;
    const int len = row_len(__ldg(nnb + p));
    for (int e = threadIdx.x & 31; e < len; e += 32) visit(__ldg(sidx + __ldg(row + e)));
}

__device__ __forceinline__ int warp_id_global() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int warps_total() { return (gridDim.x * blockDim.x) >> 5; }

// Counts over the masked neighbour types; s_i and s'_i from the particle's own type.
__global__ void __launch_bounds__(SC_TPB) k_tcount(int n, Geom g, P64* __restrict__ pos, SuperCaps cp, GroupAux aux,
                                                   const uint16_t* __restrict__ nbr, const int* __restrict__ nnb,
                                                   const int* __restrict__ id, TypedDev t,
                                                   double* __restrict__ ds_out, double2* __restrict__ sA,
                                                   CountOut out, Status* st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rebuild = 0;
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const P64 pi = pos[p];
        const int ti = t.tsort[p];
        double acc = 0.0;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            const int k = ti * t.T + t.tsort[j];
            if (!t.mask[k]) return;
            const Coef& c = t.pc[k];
            const double r2 = r2_d<ModeF64>(pi, pos[j], g);
            if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
        });
        acc = group_sum(acc, 32);
        const Coef& own = t.pc[ti * t.T + ti];
        const double s = omega_d(acc, own.fd, own.fd + 1.0), ds = domega_d(acc, own.fd, own.fd + 1.0);
        if ((threadIdx.x & 31) == 0) {
            ds_out[p] = ds;
            sA[p] = make_double2(s, 0.0);
            put_w(pos + p, s);
            if (out.n_out) out.n_out[id[p]] = acc;
            if (ds != 0.0 && out.in_window) atomicAdd((unsigned long long*)out.in_window, 1ull);
        }
    }
}

// A_i = s'_i sum_j s_j V_a^{ij} for the particles inside their switching window.
__global__ void __launch_bounds__(SC_TPB) k_tchain(int n, Geom g, const P64* __restrict__ pos, SuperCaps cp,
                                                   GroupAux aux, const uint16_t* __restrict__ nbr,
                                                   const int* __restrict__ nnb, TypedDev t,
                                                   const double* __restrict__ ds, double2* __restrict__ sA,
                                                   Status* st)
{
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const double dsi = ds[p];
        if (dsi == 0.0) continue;  // uniform over the warp
        const P64 pi = pos[p];
        const int ti = t.tsort[p];
        double acc = 0.0;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            const Coef& c = t.pc[ti * t.T + t.tsort[j]];
            const P64 pj = pos[j];
            const double r2 = r2_d<ModeF64>(pi, pj, g);
            if (r2 > c.rr2 && r2 < c.ra2) acc += get_s(pj) * Va_d(sqrt(r2), c);
        });
        acc = group_sum(acc, 32);
        if ((threadIdx.x & 31) == 0) sA[p].y = dsi * acc;
    }
}

// g_ij / r of one pair (no bond term).
__device__ __forceinline__ double typed_gr(double r2, int ti, int tj, double si, double Ai, double sj, double Aj,
                                           const TypedDev& t)
{
    const int k = ti * t.T + tj;
    const Coef& c = t.pc[k];
    if (r2 >= c.rc2) return 0.0;
    double gr = dVr_over_r_d(r2, c);
    const double r = sqrt(r2);
    if (r > 0.0) {
        const double chain = (t.mask[k] ? Ai : 0.0) + (t.mask[tj * t.T + ti] ? Aj : 0.0);
        gr += (si * sj * dVa_d(r, c) + chain * domega_d(r, c.r_l, c.r_h)) / r;
    }
    return gr;
}

// Visits the bonds of sorted particle p: bond(q) with q the partner's sorted index.
template <class Visit>
__device__ __forceinline__ void typed_bonds(int p, const int* __restrict__ id, const TypedDev& t, Visit&& bond)
{
    const int o = id[p];
    for (long long k = t.bptr[o]; k < t.bptr[o + 1]; ++k) bond(t.inv[t.bto[k]]);
}

// Forces of every particle (pairs and bonds) into its force slot.
__global__ void __launch_bounds__(SC_TPB) k_tforce(int n, Geom g, const P64* __restrict__ pos, SuperCaps cp,
                                                   GroupAux aux, const uint16_t* __restrict__ nbr,
                                                   const int* __restrict__ nnb, const int* __restrict__ id,
                                                   TypedDev t, const double2* __restrict__ sA, Status* st)
{
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const P64 pi = pos[p];
        const int ti = t.tsort[p];
        const double2 sai = sA[p];
        double fx = 0.0, fy = 0.0, fz = 0.0;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            double dx, dy, dz;
            ModeF64::delta64(pi, pos[j], g, dx, dy, dz);
            const double2 saj = sA[j];
            const double r2 = __fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)));
            const double gr = typed_gr(r2, ti, t.tsort[j], sai.x, sai.y, saj.x, saj.y, t);
            fx -= gr * dx;
            fy -= gr * dy;
            fz -= gr * dz;
        });
        fx = group_sum(fx, 32);
        fy = group_sum(fy, 32);
        fz = group_sum(fz, 32);
        if ((threadIdx.x & 31) == 0) {
            typed_bonds(p, id, t, [&](int q) {
                double dx, dy, dz;
                ModeF64::delta64(pi, pos[q], g, dx, dy, dz);
                const double r = sqrt(__fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz))));
                if (r > 0.0) {
                    const double gr = t.kb * (r - t.r0) / r;
                    fx -= gr * dx;
                    fy -= gr * dy;
                    fz -= gr * dz;
                }
            });
            static_cast<F64x4*>(aux.fcore)[p] = F64x4{fx, fy, fz, 0.0};
        }
    }
}

// ---------------------------------------------------------------- FP32-split walks
// Counts over the masked neighbour types in fixed point (the single-type
// split's arithmetic with the pair's own coefficients); s_i and s'_i from the
// particle's own type.  resid holds the packed residual bits of the positions (window pairs).
__global__ void __launch_bounds__(SC_TPB) k_tcount32(int n, Geom g, int4* __restrict__ pos, SuperCaps cp,
                                                     GroupAux aux, const uint16_t* __restrict__ nbr,
                                                     const int* __restrict__ nnb, const int* __restrict__ id,
                                                     TypedDev t, const int* __restrict__ resid,
                                                     float* __restrict__ ds_out, float2* __restrict__ sA,
                                                     CountOut out, Status* st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rebuild = 0;
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const int4 pi = pos[p];
        const int ri = __ldg(resid + p);
        const int ti = t.tsort[p];
        int full = 0;
        unsigned long long q = 0;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            const int k = ti * t.T + t.tsort[j];
            if (!t.mask[k]) return;
            const Coef& c = t.pc[k];
            const int4 pj = pos[j];
            const unsigned long long r2 = r2_fix(pi, pj);
            if (r2 >= c.rh2_fix) return;
            if (r2 <= c.rl2_fix) {
                ++full;
                return;
            }
            // omega has zero slope at both ends of the window: a pair the finer separation
            // moves across r_l or r_h changes n_i by O(dr^2)
            const unsigned long long rf = r2_fine(pi, ri, pj, __ldg(resid + j), r2);
            if (rf <= c.rl2_fix) q += 2147483648ull;
            else if (rf < c.rh2_fix) q += window_weight_fix31(rf, rf - c.rl2_fix, c.rl_s, c.w_s);
        });
        full = group_sum(full, 32);
        q = group_sum(q, 32);
        const Coef& own = t.pc[ti * t.T + ti];
        const long long T = ((long long)full << 31) + (long long)q - own.fd_fix;
        float sv, dsv;
        switch_from_fix(T, sv, dsv);
        if ((threadIdx.x & 31) == 0) {
            ds_out[p] = dsv;
            sA[p] = make_float2(sv, 0.0f);
            put_w(pos + p, sv);
            if (out.n_out) out.n_out[id[p]] = (double)full + (double)q * 4.656612873077393e-10;
            if (dsv != 0.0f && out.in_window) atomicAdd((unsigned long long*)out.in_window, 1ull);
        }
    }
}

// A_i = s'_i sum_j s_j V_a^{ij} (FP32) for the particles inside their window.
__global__ void __launch_bounds__(SC_TPB) k_tchain32(int n, Geom g, const int4* __restrict__ pos, SuperCaps cp,
                                                     GroupAux aux, const uint16_t* __restrict__ nbr,
                                                     const int* __restrict__ nnb, TypedDev t,
                                                     const float* __restrict__ ds, float2* __restrict__ sA,
                                                     Status* st)
{
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const float dsi = ds[p];
        if (dsi == 0.0f) continue;  // uniform over the warp
        const int4 pi = pos[p];
        const int ti = t.tsort[p];
        float acc = 0.0f;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            const Coef& c = t.pc[ti * t.T + t.tsort[j]];
            const int4 pj = pos[j];
            const unsigned long long r2i = r2_fix(pi, pj);
            if (r2i > c.rr2_fix && r2i < c.ra2_fix) {
                const float r2 = u64_to_float(r2i) * g.s32sq;
                const float r = r2 * rsqrtf(r2);
                const float uu = __fdividef(s64_to_float((long long)r2i - (long long)c.rm2_fix) * c.s2hinv, r + c.rmf);
                const float qq = 1.0f - uu * uu;
                acc = __fmaf_rn(get_s(pj), -c.Eaf * qq * qq, acc);
            }
        });
        acc = group_sum(acc, 32);
        if ((threadIdx.x & 31) == 0) sA[p].y = dsi * acc;
    }
}

// Forces of every particle (pairs and bonds, FP32) into its force slot.  A
// pair's chain-rule factor is mask[t_i][t_j] A_i + mask[t_j][t_i] A_j.
__global__ void __launch_bounds__(SC_TPB) k_tforce32(int n, Geom g, const int4* __restrict__ pos, SuperCaps cp,
                                                     GroupAux aux, const uint16_t* __restrict__ nbr,
                                                     const int* __restrict__ nnb, const int* __restrict__ id,
                                                     TypedDev t, const float2* __restrict__ sA, Status* st)
{
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const int4 pi = pos[p];
        const int ti = t.tsort[p];
        const float2 sai = sA[p];
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            const int tj = t.tsort[j];
            const int k = ti * t.T + tj;
            const float2 saj = sA[j];
            pair_f32(pi, sai.x, t.mask[k] ? sai.y : 0.0f, pos[j], saj.x, t.mask[tj * t.T + ti] ? saj.y : 0.0f,
                     t.pc[k], g, fx, fy, fz);
        });
        fx = group_sum(fx, 32);
        fy = group_sum(fy, 32);
        fz = group_sum(fz, 32);
        if ((threadIdx.x & 31) == 0) {
            typed_bonds(p, id, t, [&](int q) {
                const int4 pq = pos[q];
                const float dx = (float)(pi.x - pq.x) * g.s32, dy = (float)(pi.y - pq.y) * g.s32,
                            dz = (float)(pi.z - pq.z) * g.s32;
                const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
                if (r2 > 0.0f) {
                    const float rinv = rsqrtf(r2);
                    const float gr = (float)t.kb * (r2 * rinv - (float)t.r0) * rinv;
                    fx = __fmaf_rn(-gr, dx, fx);
                    fy = __fmaf_rn(-gr, dy, fy);
                    fz = __fmaf_rn(-gr, dz, fz);
                }
            });
            static_cast<float4*>(aux.fcore)[p] = make_float4(fx, fy, fz, 0.0f);
        }
    }
}

// ---------------------------------------------------------------- FP64 energy walks (either mode)
// FP64 counts, s and s' of every particle from the positions of mode M, into
// sd (s, s') and, on request, n_out (caller order).
template <class M>
__global__ void __launch_bounds__(SC_TPB) k_tcount_e(int n, Geom g, const typename M::pos_t* __restrict__ pos,
                                                     SuperCaps cp, GroupAux aux, const uint16_t* __restrict__ nbr,
                                                     const int* __restrict__ nnb, const int* __restrict__ id,
                                                     TypedDev t, double2* __restrict__ sd, double* __restrict__ n_out,
                                                     const Status* st)
{
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const auto pi = pos[p];
        const int ti = t.tsort[p];
        double acc = 0.0;
        typed_row(p, aux, cp, nbr, nnb, [&](int j) {
            const int k = ti * t.T + t.tsort[j];
            if (!t.mask[k]) return;
            const Coef& c = t.pc[k];
            const double r2 = r2_d<M>(pi, pos[j], g);
            if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
        });
        acc = group_sum(acc, 32);
        const Coef& own = t.pc[ti * t.T + ti];
        if ((threadIdx.x & 31) == 0) {
            sd[p] = make_double2(omega_d(acc, own.fd, own.fd + 1.0), domega_d(acc, own.fd, own.fd + 1.0));
            if (n_out) n_out[id[p]] = acc;
        }
    }
}

// FP64 (s_i, A_i) of every particle into sa, from sd.
template <class M>
__global__ void __launch_bounds__(SC_TPB) k_tchain_e(int n, Geom g, const typename M::pos_t* __restrict__ pos,
                                                     SuperCaps cp, GroupAux aux, const uint16_t* __restrict__ nbr,
                                                     const int* __restrict__ nnb, TypedDev t,
                                                     const double2* __restrict__ sd, double2* __restrict__ sa,
                                                     const Status* st)
{
    if (halted(st)) return;
    for (int p = warp_id_global(); p < n; p += warps_total()) {
        const double2 sdi = sd[p];
        double acc = 0.0;
        if (sdi.y != 0.0) {  // uniform over the warp
            const auto pi = pos[p];
            const int ti = t.tsort[p];
            typed_row(p, aux, cp, nbr, nnb, [&](int j) {
                const Coef& c = t.pc[ti * t.T + t.tsort[j]];
                const double r2 = r2_d<M>(pi, pos[j], g);
                if (r2 > c.rr2 && r2 < c.ra2) acc += sd[j].x * Va_d(sqrt(r2), c);
            });
            acc = group_sum(acc, 32);
        }
        if ((threadIdx.x & 31) == 0) sa[p] = make_double2(sdi.x, sdi.y * acc);
    }
}

// U and W: half of every pair and bond from each end, one partial sum per
// block (the grid has nb blocks, nb <= the partial arrays' length), then
// k_reduce_final.  Pairs with r < r_c of their types are counted from each end.
// sA holds FP64 (s_i, A_i).
template <class M>
__global__ void __launch_bounds__(SC_TPB) k_tenergy(int n, Geom g, const typename M::pos_t* __restrict__ pos,
                                                    SuperCaps cp, GroupAux aux, const uint16_t* __restrict__ nbr,
                                                    const int* __restrict__ nnb, const int* __restrict__ id,
                                                    TypedDev t, const double2* __restrict__ sA,
                                                    double* __restrict__ partial, long long* __restrict__ ppairs,
                                                    const Status* st)
{
    __shared__ double se[SC_TPB / 32], sw[SC_TPB / 32];
    __shared__ long long sp[SC_TPB / 32];
    double e = 0.0, w = 0.0;
    long long np = 0;
    if (!halted(st)) {
        for (int p = warp_id_global(); p < n; p += warps_total()) {
            const auto pi = pos[p];
            const int ti = t.tsort[p];
            const double2 sai = sA[p];
            double ep = 0.0, wp = 0.0;
            long long npp = 0;
            typed_row(p, aux, cp, nbr, nnb, [&](int j) {
                const auto pj = pos[j];
                const double r2 = r2_d<M>(pi, pj, g);
                const int tj = t.tsort[j];
                const Coef& c = t.pc[ti * t.T + tj];
                if (r2 >= c.rc2) return;
                const double2 saj = sA[j];
                const double r = sqrt(r2);
                ep += 0.5 * (Vr_d(r2, c) + sai.x * saj.x * Va_d(r, c));
                wp += 0.5 * (-typed_gr(r2, ti, tj, sai.x, sai.y, saj.x, saj.y, t) * r2);
                ++npp;
            });
            if ((threadIdx.x & 31) == 0) {
                typed_bonds(p, id, t, [&](int q) {
                    double dx, dy, dz;
                    M::delta64(pi, pos[q], g, dx, dy, dz);
                    const double r = sqrt(__fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)))), u = r - t.r0;
                    ep += 0.5 * (0.5 * t.kb * u * u);
                    wp += 0.5 * (-t.kb * u * r);
                });
            }
            e += ep;
            w += wp;
            np += npp;
        }
    }
    e = group_sum(e, 32);
    w = group_sum(w, 32);
    np = group_sum(np, 32);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        se[wid] = e;
        sw[wid] = w;
        sp[wid] = np;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double E = 0.0, Wv = 0.0;
        long long P = 0;
        for (int k = 0; k < SC_TPB / 32; ++k) {
            E += se[k];
            Wv += sw[k];
            P += sp[k];
        }
        partial[2 * blockIdx.x] = E;
        partial[2 * blockIdx.x + 1] = Wv;
        ppairs[blockIdx.x] = P;
    }
}

}  // namespace vbc
