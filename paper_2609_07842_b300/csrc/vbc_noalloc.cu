// vbc_noalloc.cu -- a VBC force evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's allocator or memory budget, real-time loops that must not take
// an allocation's latency or risk its failure, and plug-ins that are handed
// device buffers but are not allowed to create their own.  For them,
// vbc_compute_forces_noalloc() evaluates counts and forces for one small
// system with no vbc_system object: the caller passes device inputs and
// outputs, and the scratch that the three passes hand to one another (fixed-
// point positions, the switch s and chain term A, and s') lives in one
// file-scope __device__ array of fixed size.  Every GPU that loads the
// library holds that array until the process exits.
//
// The passes walk all pairs (tiles of 128 positions through shared memory)
// instead of a neighbour list, because a list would need scratch that grows
// with the density.  The arithmetic is the FP32-split arithmetic of the main
// path: 32-bit fixed-point positions, exact integer squared separations,
// integer counts plus 2^-31 fixed-point window weights, FP32 pair terms.
#include "vbc.h"
#include "vbc_device.cuh"

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

constexpr int NA_TPB = 128;

// Scratch layout (per particle): int4 fixed-point position, float2 (s, A), float s'.
constexpr size_t NA_POS_BYTES = (size_t)VBC_NOALLOC_MAX_N * sizeof(int4);
constexpr size_t NA_SA_BYTES = (size_t)VBC_NOALLOC_MAX_N * sizeof(float2);
constexpr size_t NA_DS_BYTES = (size_t)VBC_NOALLOC_MAX_N * sizeof(float);
constexpr size_t NA_SCRATCH_BYTES = NA_POS_BYTES + NA_SA_BYTES + NA_DS_BYTES;

static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

// Device address of na_scratch, looked up once per device (host code cannot
// use the symbol itself: on the host it names a stand-in, not device memory).
constexpr int NA_MAX_DEVICES = 64;
unsigned char* na_scratch_ptr[NA_MAX_DEVICES] = {};
std::mutex na_mutex;

}  // namespace

// Records the message that vbc_last_error() returns (defined with the rest of
// the C ABI; hidden from the library's exported symbols).
namespace vbc_detail {
int set_error(int code, const char* msg);
}

namespace {

int na_fail(int code, const char* msg) { return vbc_detail::set_error(code, msg); }

struct NAConst {
    float s32, s32sq;
    double inv32;
    vbc::Coef c;
};

__global__ void __launch_bounds__(NA_TPB) k_na_load(int n, const double* __restrict__ pos, double inv32,
                                                    int4* __restrict__ p32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p32[i] = make_int4((int)(uint32_t)__double2ll_rn(pos[3 * (size_t)i + 0] * inv32),
                       (int)(uint32_t)__double2ll_rn(pos[3 * (size_t)i + 1] * inv32),
                       (int)(uint32_t)__double2ll_rn(pos[3 * (size_t)i + 2] * inv32), 0);
}

// Pass 1 over all pairs: n_i, then s_i and s'_i (Eqs. counter, Psidelta).
__global__ void __launch_bounds__(NA_TPB) k_na_count(int n, NAConst k, const int4* __restrict__ p32,
                                                     float2* __restrict__ sA, float* __restrict__ ds,
                                                     double* __restrict__ counts)
{
    __shared__ int4 tile[NA_TPB];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int4 pi = i < n ? p32[i] : make_int4(0, 0, 0, 0);
    unsigned full = 0;
    unsigned long long q = 0;
    for (int base = 0; base < n; base += NA_TPB) {
        __syncthreads();
        if (base + (int)threadIdx.x < n) tile[threadIdx.x] = p32[base + threadIdx.x];
        __syncthreads();
        const int m = min(NA_TPB, n - base);
        for (int u = 0; u < m; ++u) {
            if (base + u == i) continue;
            const int4 pj = tile[u];
            const int dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                          (unsigned long long)((long long)dy * dy) +
                                          (unsigned long long)((long long)dz * dz);
            if (r2 < k.c.rh2_fix) {
                if (r2 <= k.c.rl2_fix) ++full;
                else q += vbc::window_weight_fix31(r2, r2 - k.c.rl2_fix, k.c.rl_s, k.c.w_s);
            }
        }
    }
    if (i >= n) return;
    const long long T = ((long long)full << 31) + (long long)q - k.c.fd_fix;
    float s = 1.0f, d = 0.0f;
    if (T >= 2147483648LL) {
        s = 0.0f;
    } else if (T > 0) {
        const float t = (float)T * 4.656612873077393e-10f;
        const float qq = 1.0f - t * t;
        s = qq * qq;
        d = -4.0f * t * qq;
    }
    sA[i] = make_float2(s, 0.0f);
    ds[i] = d;
    if (counts) counts[i] = (double)full + (double)q * 4.656612873077393e-10;
}

// Chain-rule pass over all pairs: A_i = s'_i sum_j s_j V_a(r_ij).
__global__ void __launch_bounds__(NA_TPB) k_na_chain(int n, NAConst k, const int4* __restrict__ p32,
                                                     float2* __restrict__ sA, const float* __restrict__ ds)
{
    __shared__ int4 tile[NA_TPB];
    __shared__ float stile[NA_TPB];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int4 pi = i < n ? p32[i] : make_int4(0, 0, 0, 0);
    const float dsi = i < n ? ds[i] : 0.0f;
    float acc = 0.0f;
    for (int base = 0; base < n; base += NA_TPB) {
        __syncthreads();
        if (base + (int)threadIdx.x < n) {
            tile[threadIdx.x] = p32[base + threadIdx.x];
            stile[threadIdx.x] = sA[base + threadIdx.x].x;
        }
        __syncthreads();
        if (dsi == 0.0f) continue;
        const int m = min(NA_TPB, n - base);
        for (int u = 0; u < m; ++u) {
            if (base + u == i) continue;
            const int4 pj = tile[u];
            const float dx = (float)(pi.x - pj.x) * k.s32, dy = (float)(pi.y - pj.y) * k.s32,
                        dz = (float)(pi.z - pj.z) * k.s32;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > k.c.rr2f && r2 < k.c.ra2f) {
                const float uu = (sqrtf(r2) - k.c.rmf) * k.c.hinvf;
                const float qq = 1.0f - uu * uu;
                acc += stile[u] * (-k.c.Eaf * qq * qq);
            }
        }
    }
    __syncthreads();
    if (i < n && dsi != 0.0f) sA[i].y = dsi * acc;
}

// Pass 2 over all pairs: F_i (Eqs. Vhat, softcore with the chain-rule term).
__global__ void __launch_bounds__(NA_TPB) k_na_force(int n, NAConst k, const int4* __restrict__ p32,
                                                     const float2* __restrict__ sA, double* __restrict__ F)
{
    __shared__ int4 tile[NA_TPB];
    __shared__ float2 satile[NA_TPB];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int4 pi = i < n ? p32[i] : make_int4(0, 0, 0, 0);
    const float2 sai = i < n ? sA[i] : make_float2(0.0f, 0.0f);
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    for (int base = 0; base < n; base += NA_TPB) {
        __syncthreads();
        if (base + (int)threadIdx.x < n) {
            tile[threadIdx.x] = p32[base + threadIdx.x];
            satile[threadIdx.x] = sA[base + threadIdx.x];
        }
        __syncthreads();
        const int m = min(NA_TPB, n - base);
        for (int u = 0; u < m; ++u) {
            if (base + u == i) continue;
            const int4 pj = tile[u];
            const float dx = (float)(pi.x - pj.x) * k.s32, dy = (float)(pi.y - pj.y) * k.s32,
                        dz = (float)(pi.z - pj.z) * k.s32;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= k.c.rc2f) continue;
            const float2 saj = satile[u];
            const float rinv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
            const float r = r2 * rinv;
            float gr = 0.0f;
            if (r2 < k.c.rr2f) gr = k.c.Er4f * (r2 * k.c.rr2invf - 1.0f);
            float gt = 0.0f;
            if (r2 > k.c.rr2f && r2 < k.c.ra2f) {
                const float uu = (r - k.c.rmf) * k.c.hinvf;
                gt = sai.x * saj.x * k.c.Ea4hf * uu * (1.0f - uu * uu);
            }
            if (r2 > k.c.rl2f && r2 < k.c.rh2f) {
                const float t = (r - k.c.rlf) * k.c.winvf;
                gt -= (sai.y + saj.y) * 4.0f * t * (1.0f - t * t) * k.c.winvf;
            }
            gr += gt * rinv;
            fx -= gr * dx;
            fy -= gr * dy;
            fz -= gr * dz;
        }
    }
    if (i >= n) return;
    F[3 * (size_t)i + 0] = fx;
    F[3 * (size_t)i + 1] = fy;
    F[3 * (size_t)i + 2] = fz;
}

int na_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return VBC_OK;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return na_fail(VBC_ERR_CUDA, buf);
}

}  // namespace

extern "C" {

int vbc_compute_forces_noalloc(int32_t n, const double* box, const double* pos, const vbc_pair_params* p,
                               double* F, double* counts, void* stream)
{
    if (n < 1 || n > VBC_NOALLOC_MAX_N) {
        char buf[160];
        snprintf(buf, sizeof(buf), "n = %d is outside [1, %d], the capacity of the static scratch", (int)n,
                 VBC_NOALLOC_MAX_N);
        return na_fail(VBC_ERR_INVALID_ARG, buf);
    }
    if (!box || !pos || !p || !F) return na_fail(VBC_ERR_INVALID_ARG, "box, pos, params and F must not be NULL");
    if (!(box[0] > 0) || !(box[0] == box[1] && box[1] == box[2]) || !std::isfinite(box[0]))
        return na_fail(VBC_ERR_INVALID_ARG, "the box must be a positive, finite cube");
    if (!(p->r_r > 0) || !(p->r_a > p->r_r) || !(p->r_l >= 0) || !(p->r_h > p->r_l) || !(p->E_r >= 0) ||
        !(p->E_a >= 0) || !std::isfinite(p->f) || !std::isfinite(p->delta) || !std::isfinite(p->r_h) ||
        !std::isfinite(p->r_a) || !std::isfinite(p->E_r) || !std::isfinite(p->E_a))
        return na_fail(VBC_ERR_INVALID_ARG, "invalid pair parameters");
    const double L = box[0];
    const double rc = std::fmax(p->r_r, std::fmax(p->r_a, p->r_h));
    if (!(2.0 * rc <= L)) return na_fail(VBC_ERR_INVALID_ARG, "the box edge must be at least twice the cut-off");

    int dev = 0;
    int rc_ = na_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc_) return rc_;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(VBC_ERR_CUDA, "device index out of range");
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_scratch_ptr[dev]) {
            void* ptr = nullptr;
            rc_ = na_check(cudaGetSymbolAddress(&ptr, na_scratch), "cudaGetSymbolAddress");
            if (rc_) return rc_;
            na_scratch_ptr[dev] = (unsigned char*)ptr;
        }
        scratch = na_scratch_ptr[dev];
    }
    int4* p32 = (int4*)scratch;
    float2* sA = (float2*)(scratch + NA_POS_BYTES);
    float* ds = (float*)(scratch + NA_POS_BYTES + NA_SA_BYTES);

    NAConst k{};
    const double s32d = L / 4294967296.0;
    k.s32 = (float)s32d;
    k.s32sq = (float)(s32d * s32d);
    k.inv32 = 4294967296.0 / L;
    {
        vbc::Coef& c = k.c;
        c.r_r = p->r_r; c.r_a = p->r_a; c.r_l = p->r_l; c.r_h = p->r_h;
        c.E_r = p->E_r; c.E_a = p->E_a; c.f = p->f; c.delta = p->delta;
        c.rr2 = p->r_r * p->r_r; c.ra2 = p->r_a * p->r_a; c.rl2 = p->r_l * p->r_l; c.rh2 = p->r_h * p->r_h;
        c.rc2 = rc * rc;
        c.rm = 0.5 * (p->r_a + p->r_r);
        c.h = 0.5 * (p->r_a - p->r_r);
        c.w = p->r_h - p->r_l;
        c.fd = p->f - p->delta;
        c.rr2f = (float)c.rr2; c.ra2f = (float)c.ra2; c.rl2f = (float)c.rl2; c.rh2f = (float)c.rh2;
        c.rc2f = (float)c.rc2;
        c.rlf = (float)p->r_l;
        c.rmf = (float)c.rm;
        c.hinvf = (float)(1.0 / c.h);
        c.winvf = (float)(1.0 / c.w);
        c.wf = (float)c.w;
        c.Er4f = (float)(4.0 * p->E_r / c.rr2);
        c.rr2invf = (float)(1.0 / c.rr2);
        c.Eaf = (float)p->E_a;
        c.Ea4hf = (float)(4.0 * p->E_a / c.h);
        const double s2 = s32d * s32d;
        c.rl2_fix = (unsigned long long)std::llround(c.rl2 / s2);
        c.rh2_fix = (unsigned long long)std::llround(c.rh2 / s2);
        const double rl_s = p->r_l / s32d, w_s = c.w / s32d;
        c.rl_s.hi = (float)rl_s;
        c.rl_s.lo = (float)(rl_s - (double)c.rl_s.hi);
        c.w_s.hi = (float)w_s;
        c.w_s.lo = (float)(w_s - (double)c.w_s.hi);
        const double fd = std::fmin(std::fmax(c.fd, -1.0e9), 1.0e9);
        double fi = std::floor(fd);
        long long frac = std::llround((fd - fi) * 2147483648.0);
        if (frac >= 2147483648LL) {
            fi += 1.0;
            frac -= 2147483648LL;
        }
        c.fd_int = (long long)fi;
        c.fd_frac_fix = frac;
        c.fd_fix = c.fd_int * 2147483648LL + frac;
    }

    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (n + NA_TPB - 1) / NA_TPB;
    k_na_load<<<nb, NA_TPB, 0, st>>>(n, pos, k.inv32, p32);
    k_na_count<<<nb, NA_TPB, 0, st>>>(n, k, p32, sA, ds, counts);
    k_na_chain<<<nb, NA_TPB, 0, st>>>(n, k, p32, sA, ds);
    k_na_force<<<nb, NA_TPB, 0, st>>>(n, k, p32, sA, F);
    rc_ = na_check(cudaGetLastError(), "kernel launch");
    if (rc_) return rc_;
    return na_check(cudaStreamSynchronize(st), "cudaStreamSynchronize");
}

}  // extern "C"
