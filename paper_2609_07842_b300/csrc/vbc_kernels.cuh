// vbc_kernels.cuh -- CUDA kernels of the VBC path (sm_103a).
//
// Particles are stored in Morton order of their cells.  Kernels that walk
// neighbour lists run in blocks of TPB = 128 consecutive particles, and each
// block first copies the union of its particles' 27-cell neighbourhoods (a
// set of whole cells, i.e. contiguous runs of the sorted arrays) into shared
// memory: the staging.  Neighbour lists store 16-bit indices into that
// staging, so a pass reads 2 bytes per list entry from HBM and serves every
// neighbour lookup from shared memory.
//
// One MD step:
//   rebuild (only when a particle moved more than skin/2 since the last build):
//     k_bin -> k_scan_sums -> k_scan_apply -> k_scatter -> k_cellsort ->
//     k_permute -> k_copyback -> k_stage_table -> k_nlist
//   k_count   pass 1: n_i, s_i, s'_i                        (Eqs. counter, Psidelta)
//   k_chain   A_i = s'_i sum_j s_j V_a(r_ij), window particles only
//   k_force   pass 2: F_i, fused with the BAOAB update of the state
//   k_count_e, k_chain_e, k_energy   FP64 U, W and pair count (on request only)
// The rebuild kernels read a device flag and return at once when no rebuild
// is due, so the host never waits on the device between steps.  Every pass
// walks a full (both-direction) list, one thread per particle, and
// accumulates without atomics, so results do not depend on scheduling.
#pragma once

#include "vbc_device.cuh"

namespace vbc {

constexpr int TPB = 128;          // threads per block of the per-particle kernels
constexpr int SCAN_CHUNK = 2048;  // cells per block in the two-pass scan
constexpr int SCAN_TPB = 256;
constexpr int MAX_CELL = 512;     // a denser cell means the system has collapsed
constexpr int HASH_SIZE = 4096;   // open-addressing set of a block's neighbour cells

enum Epilogue { EPI_FORCE = 0, EPI_START = 1, EPI_FINISH = 2, EPI_FINISH_START = 3 };

// ================================================================ rebuild: sort by cell
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
        st->max_stage = 0;
        st->max_stage_cells = 0;
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

// Gathers the state (8-byte words: positions and velocities of either mode),
// the original index and the fixed-point position into sorted order.
template <class M>
__global__ void __launch_bounds__(TPB) k_permute(int n, const int* __restrict__ order,
                                                 const unsigned long long* __restrict__ x,
                                                 const unsigned long long* __restrict__ v,
                                                 const int* __restrict__ id,
                                                 const typename M::pos_t* __restrict__ pos,
                                                 unsigned long long* __restrict__ xt,
                                                 unsigned long long* __restrict__ vt, int* __restrict__ idt,
                                                 typename M::pos_t* __restrict__ post, const Status* st)
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
__global__ void __launch_bounds__(TPB) k_copyback(int n, const unsigned long long* __restrict__ xt,
                                                  const unsigned long long* __restrict__ vt,
                                                  const int* __restrict__ idt,
                                                  const typename M::pos_t* __restrict__ post,
                                                  unsigned long long* __restrict__ x, unsigned long long* __restrict__ v,
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

// ================================================================ staging
// A block's staging is a list of runs: maximal sequences of cells with
// consecutive Morton ranks, i.e. contiguous ranges of the sorted particle
// arrays.  Run k of block b starts at sorted particle base[b*cmax + k], holds
// off[b*(cmax+1) + k + 1] - off[b*(cmax+1) + k] particles at that staging
// offset, and begins with the cell of rank rank[b*cmax + k].
struct StageTable {
    int* base;
    int* off;
    int* rank;
    int* n;    // runs per block
    int cmax;  // capacity in cells (and runs) per block
    int smax;  // capacity in staged particles per block
};

// A list: near entries (closer than max(r_r, r_l) at the build) in rows
// 0..nn-1 from the front, far entries (up to r_list) in rows cap-1, cap-2, ...
// from the back, column-major nbr[row * n + i]; nnb[i] = nn | nf << 16.
struct ListRef {
    const uint16_t* nbr;
    const int* nnb;
    int cap;
};

template <class F>
__device__ __forceinline__ void for_entries(const ListRef& L, int n, int i, int nn, int nf, F&& f)
{
#pragma unroll 4
    for (int t = 0; t < nn; ++t) f((int)__ldg(L.nbr + (size_t)t * n + i));
#pragma unroll 4
    for (int t = 0; t < nf; ++t) f((int)__ldg(L.nbr + (size_t)(L.cap - 1 - t) * n + i));
}

// Loads block b's run table (base, off) into shared memory; returns the
// number of staged particles.  s_base and s_off hold cmax and cmax + 1 ints.
__device__ __forceinline__ int load_runs(const StageTable& tb, int b, int* s_base, int* s_off, int& R)
{
    R = tb.n[b];
    for (int k = threadIdx.x; k < R; k += blockDim.x) s_base[k] = tb.base[(size_t)b * tb.cmax + k];
    for (int k = threadIdx.x; k <= R; k += blockDim.x) s_off[k] = tb.off[(size_t)b * (tb.cmax + 1) + k];
    __syncthreads();
    return s_off[R];
}

// Copies every staged particle: copy(staging index, sorted index), one warp per run.
template <class F>
__device__ __forceinline__ void stage_runs(const int* s_base, const int* s_off, int R, F&& copy)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < R; k += (int)(blockDim.x >> 5)) {
        const int b = s_base[k], o = s_off[k], len = s_off[k + 1] - o;
        for (int l = lane; l < len; l += 32) copy(o + l, b + l);
    }
}

// Dynamic shared memory of the pass kernels: base[cmax] | off[cmax+1] | staged arrays.
__host__ __device__ inline size_t stage_header_bytes(int cmax) { return (((size_t)(2 * cmax + 1) * 4) + 15) & ~(size_t)15; }
// ... of k_stage_table: hash[HASH_SIZE] | cells[cmax] | starts[cmax+1]
__host__ __device__ inline size_t stage_table_smem(int cmax) { return (size_t)(HASH_SIZE + 2 * cmax + 1) * 4; }
// ... of k_nlist: base[cmax] | off[cmax+1] | rank[cmax] | staged positions
__host__ __device__ inline size_t nlist_header_bytes(int cmax) { return (((size_t)(3 * cmax + 1) * 4) + 15) & ~(size_t)15; }

// Near (0), far (1) or beyond the list radius (-1), from exact integer squared
// separations in the FP32 mode.
struct ListParams {
    unsigned long long rlist2_fix, near2_fix;
    double rlist2, near2;
};
template <class M>
struct ListTest;
template <>
struct ListTest<ModeF32> {
    __device__ __forceinline__ static int cls(const int4& a, const int4& b, const Geom&, const ListParams& lp)
    {
        const int dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                      (unsigned long long)((long long)dy * dy) +
                                      (unsigned long long)((long long)dz * dz);
        if (r2 >= lp.rlist2_fix) return -1;
        return r2 < lp.near2_fix ? 0 : 1;
    }
};
template <>
struct ListTest<ModeF64> {
    __device__ __forceinline__ static int cls(const P64& a, const P64& b, const Geom& g, const ListParams& lp)
    {
        double dx, dy, dz;
        ModeF64::delta64(a, b, g, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= lp.rlist2) return -1;
        return r2 < lp.near2 ? 0 : 1;
    }
};

// Neighbour cell d (0..26) of cell (x, y, z), periodic.
__device__ __forceinline__ int neighbour_cell_lin(int x, int y, int z, int d, const Geom& g)
{
    x += d % 3 - 1;
    y += (d / 3) % 3 - 1;
    z += d / 9 - 1;
    x = x < 0 ? x + g.nc[0] : (x >= g.nc[0] ? x - g.nc[0] : x);
    y = y < 0 ? y + g.nc[1] : (y >= g.nc[1] ? y - g.nc[1] : y);
    z = z < 0 ? z + g.nc[2] : (z >= g.nc[2] ? z - g.nc[2] : z);
    return (z * g.nc[1] + y) * g.nc[0] + x;
}

// ================================================================ rebuild: staging tables
// For each block of TPB sorted particles: the set of cells in the
// 27-neighbourhoods of its particles' cells (open-addressing hash in shared
// memory), sorted by Morton rank and merged into runs of consecutive ranks,
// with staging offsets; written to the global run table.
template <class M>
__global__ void __launch_bounds__(TPB) k_stage_table(int n, Geom g, const typename M::pos_t* __restrict__ pos,
                                                     const int* __restrict__ morton_rank,
                                                     const int* __restrict__ rank_to_lin,
                                                     const int* __restrict__ cell_start, StageTable tb, Status* st)
{
    if (!st->rebuild || st->frozen || st->crowded) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* hash = (int*)smem;
    int* cells = hash + HASH_SIZE;
    int* starts = cells + tb.cmax;
    __shared__ int s_rank[TPB];
    __shared__ int s_uniq[TPB];
    __shared__ int s_nu, s_nc;
    __shared__ int sw[TPB / 32];
    const int b = blockIdx.x;
    const int i = b * TPB + threadIdx.x;
    int rank_i = -1;
    if (i < n) {
        const int3 c = cell_of_pos<M>(pos[i], g);
        rank_i = morton_rank[(c.z * g.nc[1] + c.y) * g.nc[0] + c.x];
    }
    s_rank[threadIdx.x] = rank_i;
    for (int h = threadIdx.x; h < HASH_SIZE; h += TPB) hash[h] = -1;
    if (threadIdx.x == 0) {
        s_nu = 0;
        s_nc = 0;
    }
    __syncthreads();
    // unique cells of the block (ranks ascend along the sorted particles)
    if (i < n && (threadIdx.x == 0 || s_rank[threadIdx.x - 1] != rank_i)) s_uniq[atomicAdd(&s_nu, 1)] = rank_i;
    __syncthreads();
    const int U = s_nu;
    for (int t = threadIdx.x; t < 27 * U; t += TPB) {
        const int u = t / 27, d = t - 27 * u;
        const int lin = rank_to_lin[s_uniq[u]];
        const int r = morton_rank[neighbour_cell_lin(lin % g.nc[0], (lin / g.nc[0]) % g.nc[1],
                                                     lin / (g.nc[0] * g.nc[1]), d, g)];
        unsigned h = ((unsigned)r * 2654435761u) & (HASH_SIZE - 1);
        for (int probe = 0; probe < HASH_SIZE; ++probe) {
            const int old = atomicCAS(&hash[h], -1, r);
            if (old == -1) {
                const int idx = atomicAdd(&s_nc, 1);
                if (idx < tb.cmax) cells[idx] = r;
                break;
            }
            if (old == r) break;
            h = (h + 1) & (HASH_SIZE - 1);
        }
    }
    __syncthreads();
    const int S = s_nc;
    if (S > tb.cmax) {
        if (threadIdx.x == 0) {
            atomicMax(&st->max_stage_cells, S);
            st->stage_overflow = 1;
            st->frozen_iter = (int)st->iter;
        }
        return;
    }
    // sort the cells by rank (bitonic over the next power of two, padded)
    int P = 1;
    while (P < S) P <<= 1;
    for (int k = S + threadIdx.x; k < P; k += TPB) cells[k] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += TPB) {
                const int o = t ^ j;
                if (o > t) {
                    const int a = cells[t], c = cells[o];
                    if ((a > c) == ((t & k) == 0)) {
                        cells[t] = c;
                        cells[o] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // runs of consecutive ranks: start positions, consecutive cells per thread
    const int per = (S + TPB - 1) / TPB;
    const int k0 = min(S, (int)threadIdx.x * per), k1 = min(S, ((int)threadIdx.x + 1) * per);
    int nstart = 0;
    for (int k = k0; k < k1; ++k) nstart += (k == 0 || cells[k] != cells[k - 1] + 1);
    int R;
    int r = block_exclusive_scan<TPB>(nstart, sw, R);
    for (int k = k0; k < k1; ++k)
        if (k == 0 || cells[k] != cells[k - 1] + 1) starts[r++] = k;
    if (threadIdx.x == 0) starts[R] = S;
    __syncthreads();
    // staging offsets of the runs
    const int rper = (R + TPB - 1) / TPB;
    const int q0 = min(R, (int)threadIdx.x * rper), q1 = min(R, ((int)threadIdx.x + 1) * rper);
    int len = 0;
    for (int q = q0; q < q1; ++q)
        len += cell_start[cells[starts[q + 1] - 1] + 1] - cell_start[cells[starts[q]]];
    int total;
    int o = block_exclusive_scan<TPB>(len, sw, total);
    for (int q = q0; q < q1; ++q) {
        const int first = cells[starts[q]];
        const int bq = cell_start[first];
        tb.base[(size_t)b * tb.cmax + q] = bq;
        tb.rank[(size_t)b * tb.cmax + q] = first;
        tb.off[(size_t)b * (tb.cmax + 1) + q] = o;
        o += cell_start[cells[starts[q + 1] - 1] + 1] - bq;
    }
    if (threadIdx.x == 0) {
        tb.off[(size_t)b * (tb.cmax + 1) + R] = total;
        tb.n[b] = R;
        atomicMax(&st->max_stage, total);
        atomicMax(&st->max_stage_cells, S);
        if (total > tb.smax) {
            st->stage_overflow = 1;
            st->frozen_iter = (int)st->iter;
        }
    }
}

// ================================================================ rebuild: lists
// Each particle's list of staged indices within r_list, near entries from the
// front and far entries from the back (so that a pass walks neighbours of
// similar distance together and the count pass can stop after the near ones).
template <class M>
__global__ void __launch_bounds__(TPB) k_nlist(int n, Geom g, const typename M::pos_t* __restrict__ pos,
                                               const int* __restrict__ morton_rank,
                                               const int* __restrict__ cell_start, StageTable tb, ListParams lp,
                                               int cap, uint16_t* __restrict__ nbr, int* __restrict__ nnb,
                                               Status* st)
{
    using pos_t = typename M::pos_t;
    // raises `overflow` itself, so it does not test it; `stage_overflow` comes from k_stage_table
    if (!st->rebuild || st->frozen || st->crowded || st->stage_overflow) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    int* s_rk = s_off + tb.cmax + 1;
    pos_t* spos = (pos_t*)(smem + nlist_header_bytes(tb.cmax));
    __shared__ int smx[TPB / 32];
    __shared__ long long ssm[TPB / 32];
    const int b = blockIdx.x;
    int R;
    load_runs(tb, b, s_base, s_off, R);
    for (int k = threadIdx.x; k < R; k += TPB) s_rk[k] = tb.rank[(size_t)b * tb.cmax + k];
    stage_runs(s_base, s_off, R, [&](int m, int j) { spos[m] = pos[j]; });
    __syncthreads();
    const int i = b * TPB + threadIdx.x;
    int count = 0;
    if (i < n) {
        const pos_t pi = pos[i];
        const int3 ci = cell_of_pos<M>(pi, g);
        // staging position of cell rank r: run with the largest first rank <= r
        auto locate = [&](int r) {
            int lo = 0, hi = R - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_rk[mid] <= r) lo = mid;
                else hi = mid - 1;
            }
            return s_off[lo] + (cell_start[r] - s_base[lo]);
        };
        const int m_self = locate(morton_rank[(ci.z * g.nc[1] + ci.y) * g.nc[0] + ci.x]) +
                           (i - cell_start[morton_rank[(ci.z * g.nc[1] + ci.y) * g.nc[0] + ci.x]]);
        int nn = 0, nf = 0;
        for (int d = 0; d < 27; ++d) {
            const int r = morton_rank[neighbour_cell_lin(ci.x, ci.y, ci.z, d, g)];
            const int o = locate(r);
            const int len = cell_start[r + 1] - cell_start[r];
            for (int m = o; m < o + len; ++m) {
                if (m == m_self) continue;
                const int cl = ListTest<M>::cls(pi, spos[m], g, lp);
                if (cl < 0) continue;
                if (nn + nf < cap) {
                    if (cl == 0) nbr[(size_t)nn * n + i] = (uint16_t)m;
                    else nbr[(size_t)(cap - 1 - nf) * n + i] = (uint16_t)m;
                }
                if (cl == 0) ++nn;
                else ++nf;
            }
        }
        count = nn + nf;
        nnb[i] = nn | (nf << 16);
        if (count > cap) {
            st->overflow = 1;
            st->frozen_iter = (int)st->iter;
        }
    }
    // block maximum and sum of the list lengths
    int mx = count;
    long long sm = count;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smx[threadIdx.x >> 5] = mx;
        ssm[threadIdx.x >> 5] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mx = smx[0];
        sm = ssm[0];
        for (int w = 1; w < TPB / 32; ++w) {
            mx = max(mx, smx[w]);
            sm += ssm[w];
        }
        atomicMax(&st->max_nnb, mx);
        atomicAdd((unsigned long long*)&st->nnb_sum, (unsigned long long)sm);
        if (blockIdx.x == 0) st->rebuilds += 1;
    }
}

// ================================================================ pass 1: counts
// FP32-split: neighbours with r <= r_l add exactly 1 (an integer); window
// neighbours add omega in 2^-31 fixed point (window_weight_fix31).  The
// threshold test t = n - (f - delta) is taken in the same fixed point, so
// s_i and s'_i carry only the error of the window terms.
// Saturation: when the near entries alone hold at least ceil(f - delta + 1)
// neighbours with r <= r_l, then n_i >= f - delta + 1 whatever the other
// entries add, so s_i = s'_i = 0 exactly and the window terms are not needed
// (unless the counts themselves are requested).
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

__device__ __forceinline__ unsigned long long r2_fix(const int4& a, const int4& b)
{
    const int dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    return (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
           (unsigned long long)((long long)dz * dz);
}

__global__ void __launch_bounds__(TPB) k_count_f32(int n, Geom g, Coef c, const int4* __restrict__ pos,
                                                   ListRef L, const int* __restrict__ id, StageTable tb,
                                                   float* __restrict__ ds_out, float2* __restrict__ sA,
                                                   CountOut out, Status* st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rebuild = 0;
    if (halted(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    int4* spos = (int4*)(smem + stage_header_bytes(tb.cmax));
    int R;
    load_runs(tb, blockIdx.x, s_base, s_off, R);
    stage_runs(s_base, s_off, R, [&](int m, int j) { spos[m] = pos[j]; });
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool win = false;
    if (i < n) {
        const int4 pi = pos[i];
        const int w = L.nnb[i];
        const int nn = w & 0xffff, nf = w >> 16;
        long long full = 0;
        for_entries(L, n, i, nn, 0, [&](int m) { full += r2_fix(pi, spos[m]) <= c.rl2_fix; });
        float s = 0.0f, ds = 0.0f;
        if (full < c.sat_full || out.n_out) {
            full = 0;
            unsigned long long q = 0;
            for_entries(L, n, i, nn, nf, [&](int m) {
                const unsigned long long r2 = r2_fix(pi, spos[m]);
                if (r2 < c.rh2_fix) {
                    if (r2 <= c.rl2_fix) ++full;
                    else q += window_weight_fix31(r2, r2 - c.rl2_fix, c.rl_s, c.w_s);
                }
            });
            const long long T = (full - c.fd_int) * 2147483648LL + (long long)q - c.fd_frac_fix;
            switch_from_fix(T, s, ds);
            if (out.n_out) out.n_out[id[i]] = (double)full + (double)q * 4.656612873077393e-10;
        }
        ds_out[i] = ds;
        sA[i] = make_float2(s, 0.0f);
        win = ds != 0.0f;
    }
    if (out.in_window) {
        const unsigned bal = __ballot_sync(0xffffffffu, win);
        if ((threadIdx.x & 31) == 0 && bal)
            atomicAdd((unsigned long long*)out.in_window, (unsigned long long)__popc(bal));
    }
}

__global__ void __launch_bounds__(TPB) k_count_f64(int n, Geom g, Coef c, const P64* __restrict__ pos, ListRef L,
                                                   const int* __restrict__ id, StageTable tb,
                                                   double* __restrict__ ds_out, double2* __restrict__ sA,
                                                   CountOut out, Status* st)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) st->rebuild = 0;
    if (halted(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    P64* spos = (P64*)(smem + stage_header_bytes(tb.cmax));
    int R;
    load_runs(tb, blockIdx.x, s_base, s_off, R);
    stage_runs(s_base, s_off, R, [&](int m, int j) { spos[m] = pos[j]; });
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool win = false;
    if (i < n) {
        const P64 pi = pos[i];
        const int w = L.nnb[i];
        double acc = 0.0;
        for_entries(L, n, i, w & 0xffff, w >> 16, [&](int m) {
            double dx, dy, dz;
            ModeF64::delta64(pi, spos[m], g, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
        });
        const double s = omega_d(acc, c.fd, c.fd + 1.0);
        const double ds = domega_d(acc, c.fd, c.fd + 1.0);
        ds_out[i] = ds;
        sA[i] = make_double2(s, 0.0);
        win = ds != 0.0;
        if (out.n_out) out.n_out[id[i]] = acc;
    }
    if (out.in_window) {
        const unsigned bal = __ballot_sync(0xffffffffu, win);
        if ((threadIdx.x & 31) == 0 && bal)
            atomicAdd((unsigned long long*)out.in_window, (unsigned long long)__popc(bal));
    }
}

// ================================================================ chain-rule pass
// A_i = s'_i sum_j s_j V_a(r_ij) for particles inside the switching window;
// blocks without such a particle return after one vote.
template <class M>
__global__ void __launch_bounds__(TPB) k_chain(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                               ListRef L, StageTable tb, const typename M::real* __restrict__ ds,
                                               typename M::real2* __restrict__ sA, const Status* st)
{
    using real = typename M::real;
    using pos_t = typename M::pos_t;
    if (halted(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const real dsi = i < n ? ds[i] : (real)0;
    if (!__syncthreads_or(dsi != (real)0)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    pos_t* spos = (pos_t*)(smem + stage_header_bytes(tb.cmax));
    real* ss = (real*)(spos + tb.smax);
    int R;
    load_runs(tb, blockIdx.x, s_base, s_off, R);
    const real* s_only = reinterpret_cast<const real*>(sA);  // s_j at even offsets
    stage_runs(s_base, s_off, R, [&](int m, int j) {
        spos[m] = pos[j];
        ss[m] = s_only[2 * (size_t)j];
    });
    __syncthreads();
    if (dsi == (real)0) return;
    const pos_t pi = pos[i];
    const int w = L.nnb[i];
    real acc = 0;
    for_entries(L, n, i, w & 0xffff, w >> 16, [&](int m) {
        if constexpr (M::fp64) {
            double dx, dy, dz;
            M::delta64(pi, spos[m], g, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > c.rr2 && r2 < c.ra2) acc += ss[m] * Va_d(sqrt(r2), c);
        } else {
            const unsigned long long r2i = r2_fix(pi, spos[m]);
            if (r2i > c.rr2_fix && r2i < c.ra2_fix) {
                const float r2 = u64_to_float(r2i) * g.s32sq;
                const float r = sqrtf(r2);
                const float u = s64_to_float((long long)r2i - (long long)c.rm2_fix) * c.s2hinv / (r + c.rmf);
                const float q = 1.0f - u * u;
                acc += ss[m] * (-c.Eaf * q * q);
            }
        }
    });
    sA[i].y = dsi * acc;
}

// ================================================================ pass 2: forces + BAOAB
struct StepArgs {
    void* x;              // [3][n] unwrapped positions (FP32 mode: int64 in units L / 2^52; FP64: double)
    void* v;              // [3][n] velocities (FP32 mode: two-float; FP64: double)
    double* F_out;        // forces in caller order [n][3], or null (EPI_FORCE)
    // FP64 mode constants
    double dt, c1, c2;    // c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT)
    // FP32 mode constants as two-floats
    f2x h;                // dt / 2
    f2x hK[3];            // dt / 2 * 2^52 / L_a: velocity -> fixed-point displacement of a half drift
    f2x c1f, c2f;
    unsigned long long seed;
    float half_skin2;     // (skin / 2)^2
};

// BAOAB update of particle i (unit mass, h = dt / 2) from its force.
// FP32 mode: the unwrapped position is an int64 in units of L / 2^52 and the
// velocity a two-float, so the update needs no FP64 instruction; each half
// drift adds the nearest integer of h v 2^52 / L.  FP64 mode: doubles.
template <class M, int EPI>
__device__ __forceinline__ void integrate(int i, int n, const Geom& g, typename M::real fx, typename M::real fy,
                                          typename M::real fz, const StepArgs& a, uint32_t pid, Status* st,
                                          typename M::pos_t* __restrict__ pos_next,
                                          const typename M::pos_t* __restrict__ xref)
{
    constexpr bool start = EPI == EPI_START || EPI == EPI_FINISH_START;
    constexpr bool finish = EPI == EPI_FINISH || EPI == EPI_FINISH_START;
    bool bad = !isfinite(fx) || !isfinite(fy) || !isfinite(fz);
    if constexpr (!M::fp64) {
        long long* X = (long long*)a.x;
        float2* V = (float2*)a.v;
        const float f3[3] = {fx, fy, fz};
        float xi[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (start) {
            const float3 z = langevin_normals(a.seed, (unsigned long long)(st->step_base + st->iter), pid);
            xi[0] = z.x;
            xi[1] = z.y;
            xi[2] = z.z;
        }
        int w[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float2 vv = V[(size_t)d * n + i];
            f2x v = {vv.x, vv.y};
            const f2x hf = f2x_mulf(a.h, f3[d]);
            if constexpr (finish) v = f2x_add(v, hf);                             // B (closes the step)
            if constexpr (start) {
                long long P = X[(size_t)d * n + i];
                v = f2x_add(v, hf);                                                // B
                P += f2x_to_ll(f2x_mul(v, a.hK[d]));                               // A
                v = f2x_add(f2x_mul(v, a.c1f), f2x_mulf(a.c2f, xi[d]));            // O
                P += f2x_to_ll(f2x_mul(v, a.hK[d]));                               // A
                X[(size_t)d * n + i] = P;
                w[d] = ModeF32::word(P);
            }
            bad |= !isfinite(v.hi);
            V[(size_t)d * n + i] = make_float2(v.hi, v.lo);
        }
        if constexpr (start) {
            const int4 pn = make_int4(w[0], w[1], w[2], 0);
            pos_next[i] = pn;
            const int4 pr = xref[i];
            const float ux = (float)(pn.x - pr.x) * g.s32, uy = (float)(pn.y - pr.y) * g.s32,
                        uz = (float)(pn.z - pr.z) * g.s32;
            if (ux * ux + uy * uy + uz * uz > a.half_skin2) st->rebuild = 1;
        }
    } else {
        double* X = (double*)a.x;
        double* V = (double*)a.v;
        const double h = 0.5 * a.dt;
        const double f3[3] = {(double)fx, (double)fy, (double)fz};
        double xs[3], vs[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xs[d] = X[(size_t)d * n + i];
            vs[d] = V[(size_t)d * n + i];
        }
        if constexpr (finish) {
#pragma unroll
            for (int d = 0; d < 3; ++d) vs[d] += h * f3[d];
        }
        if constexpr (start) {
            const double3 z = langevin_normals_d(a.seed, (unsigned long long)(st->step_base + st->iter), pid);
            const double zz[3] = {z.x, z.y, z.z};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                vs[d] += h * f3[d];
                xs[d] += h * vs[d];
                vs[d] = a.c1 * vs[d] + a.c2 * zz[d];
                xs[d] += h * vs[d];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bad |= !isfinite(xs[d]) || !isfinite(vs[d]);
            X[(size_t)d * n + i] = xs[d];
            V[(size_t)d * n + i] = vs[d];
        }
        if constexpr (start) {
            const P64 pn = ModeF64::from_x(xs[0], xs[1], xs[2], g);
            pos_next[i] = pn;
            const P64 pr = xref[i];
            float d2 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float u = (float)(int)(ModeF64::hi32(pn, d) - ModeF64::hi32(pr, d)) * (float)g.s32d[d];
                d2 += u * u;
            }
            if (d2 > a.half_skin2) st->rebuild = 1;
        }
    }
    if (bad) st->frozen = 1;
}

// Pass 2.  FP32 mode, per pair: the exact integer r^2 decides which terms can
// be nonzero (core overlap r < r_r; the well, only if s_i s_j != 0; the
// counting window, only if A_i + A_j != 0) and pairs with none of them stop
// there.  The arguments of the steep well and of the window come from exact
// integer differences r^2 - r_m^2 and r^2 - r_l^2.
template <class M, int EPI>
__global__ void __launch_bounds__(TPB) k_force(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                               ListRef L, const int* __restrict__ id, StageTable tb,
                                               const typename M::real2* __restrict__ sA,
                                               typename M::pos_t* __restrict__ pos_next,
                                               const typename M::pos_t* __restrict__ xref, StepArgs a, Status* st)
{
    using real = typename M::real;
    using real2 = typename M::real2;
    using pos_t = typename M::pos_t;
    // k_force raises `frozen` and `rebuild` itself; it tests `frozen` only through
    // halted(), which a thread of this launch changes only on the error path
    if (halted(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    pos_t* spos = (pos_t*)(smem + stage_header_bytes(tb.cmax));
    real2* ssa = (real2*)(spos + tb.smax);
    int R;
    load_runs(tb, blockIdx.x, s_base, s_off, R);
    stage_runs(s_base, s_off, R, [&](int m, int j) {
        spos[m] = pos[j];
        ssa[m] = sA[j];
    });
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const pos_t pi = pos[i];
    const real2 sai = sA[i];
    const int w = L.nnb[i];
    real fx = 0, fy = 0, fz = 0;
    for_entries(L, n, i, w & 0xffff, w >> 16, [&](int m) {
        const pos_t pj = spos[m];
        const real2 saj = ssa[m];
        if constexpr (M::fp64) {
            double dx, dy, dz;
            M::delta64(pi, pj, g, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= c.rc2) return;
            const double r = sqrt(r2);
            double gr = dVr_over_r_d(r2, c);
            if (r > 0.0) gr += (sai.x * saj.x * dVa_d(r, c) + (sai.y + saj.y) * domega_d(r, c.r_l, c.r_h)) / r;
            fx -= gr * dx;
            fy -= gr * dy;
            fz -= gr * dz;
        } else {
            const int ix = pi.x - pj.x, iy = pi.y - pj.y, iz = pi.z - pj.z;
            const unsigned long long r2i = (unsigned long long)((long long)ix * ix) +
                                           (unsigned long long)((long long)iy * iy) +
                                           (unsigned long long)((long long)iz * iz);
            const bool core = r2i < c.rr2_fix;
            const bool well = r2i > c.rr2_fix && r2i < c.ra2_fix && sai.x * saj.x != 0.0f;
            const bool chain = r2i > c.rl2_fix && r2i < c.rh2_fix && sai.y + saj.y != 0.0f;
            if (!(core || well || chain)) return;
            const float dx = (float)ix * g.s32, dy = (float)iy * g.s32, dz = (float)iz * g.s32;
            float gr = 0.0f;                                   // g / r
            if (core) gr = c.Er4f * (u64_to_float(r2i) * g.s32sq * c.rr2invf - 1.0f);
            if (well || chain) {
                const float r2 = u64_to_float(r2i) * g.s32sq;
                float rinv = rsqrtf(r2);
                rinv = rinv * __fmaf_rn(-0.5f * r2 * rinv, rinv, 1.5f);   // one Newton step
                const float r = r2 * rinv;
                float gt = 0.0f;                               // g from the well and the counts
                if (well) {
                    const float u = s64_to_float((long long)r2i - (long long)c.rm2_fix) * c.s2hinv / (r + c.rmf);
                    gt = sai.x * saj.x * c.Ea4hf * u * (1.0f - u * u);
                }
                if (chain) {
                    const float t = u64_to_float(r2i - c.rl2_fix) * c.s2winv / (r + c.rlf);
                    gt -= (sai.y + saj.y) * 4.0f * t * (1.0f - t * t) * c.winvf;
                }
                gr += gt * rinv;
            }
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
        integrate<M, EPI>(i, n, g, fx, fy, fz, a, (uint32_t)id[i], st, pos_next, xref);
    }
}

// ================================================================ FP64 energy / virial
// Requested energies are held to 1e-9 relative, which needs the switching
// factors to FP64 accuracy: the counts, s, s' and A are recomputed here in
// FP64 from the exact fixed-point separations (these kernels run only when U
// or W is asked for, never inside the step loop).  Neighbour values are read
// through each block's staging (staged index -> sorted index, kept in sj).
template <class M>
__device__ __forceinline__ int stage_pos_index(const StageTable& tb, const typename M::pos_t* __restrict__ pos,
                                               int* s_base, int* s_off, typename M::pos_t* spos, int* sj)
{
    int R;
    const int total = load_runs(tb, blockIdx.x, s_base, s_off, R);
    stage_runs(s_base, s_off, R, [&](int m, int j) {
        spos[m] = pos[j];
        sj[m] = j;
    });
    __syncthreads();
    return total;
}

template <class M>
__global__ void __launch_bounds__(TPB) k_count_e(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                 ListRef L, StageTable tb, double2* __restrict__ sd, const Status* st)
{
    using pos_t = typename M::pos_t;
    if (halted(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    pos_t* spos = (pos_t*)(smem + stage_header_bytes(tb.cmax));
    int* sj = (int*)(spos + tb.smax);
    stage_pos_index<M>(tb, pos, s_base, s_off, spos, sj);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const pos_t pi = pos[i];
    const int w = L.nnb[i];
    double acc = 0.0;
    for_entries(L, n, i, w & 0xffff, w >> 16, [&](int m) {
        double dx, dy, dz;
        M::delta64(pi, spos[m], g, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
    });
    sd[i] = make_double2(omega_d(acc, c.fd, c.fd + 1.0), domega_d(acc, c.fd, c.fd + 1.0));
}

template <class M>
__global__ void __launch_bounds__(TPB) k_chain_e(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                 ListRef L, StageTable tb, const double2* __restrict__ sd,
                                                 double* __restrict__ Ad, const Status* st)
{
    using pos_t = typename M::pos_t;
    if (halted(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    pos_t* spos = (pos_t*)(smem + stage_header_bytes(tb.cmax));
    int* sj = (int*)(spos + tb.smax);
    stage_pos_index<M>(tb, pos, s_base, s_off, spos, sj);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dsi = sd[i].y;
    if (dsi == 0.0) {
        Ad[i] = 0.0;
        return;
    }
    const pos_t pi = pos[i];
    const int w = L.nnb[i];
    double acc = 0.0;
    for_entries(L, n, i, w & 0xffff, w >> 16, [&](int m) {
        double dx, dy, dz;
        M::delta64(pi, spos[m], g, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > c.rr2 && r2 < c.ra2) acc += sd[sj[m]].x * Va_d(sqrt(r2), c);
    });
    Ad[i] = dsi * acc;
}

// Per-block partial sums of U = sum_{i<j} [V_r + s_i s_j V_a], W = sum_{i<j} -g r and
// of the number of pairs with r < r_c, each pair seen from both ends (halves).
template <class M>
__global__ void __launch_bounds__(TPB) k_energy(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                ListRef L, StageTable tb, const double2* __restrict__ sd,
                                                const double* __restrict__ Ad, double* __restrict__ partial,
                                                long long* __restrict__ ppairs, const Status* st)
{
    using pos_t = typename M::pos_t;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double se[TPB], sw[TPB];
    __shared__ long long sp[TPB];
    int* s_base = (int*)smem;
    int* s_off = s_base + tb.cmax;
    pos_t* spos = (pos_t*)(smem + stage_header_bytes(tb.cmax));
    int* sj = (int*)(spos + tb.smax);
    const bool live = !halted(st);
    if (live) stage_pos_index<M>(tb, pos, s_base, s_off, spos, sj);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, w = 0.0;
    long long pairs = 0;
    if (i < n && live) {
        const pos_t pi = pos[i];
        const double si = sd[i].x, Ai = Ad[i];
        const int nw = L.nnb[i];
        for_entries(L, n, i, nw & 0xffff, nw >> 16, [&](int m) {
            double dx, dy, dz;
            M::delta64(pi, spos[m], g, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= c.rc2) return;
            ++pairs;
            const int j = sj[m];
            const double sjv = sd[j].x, Aj = Ad[j];
            const double r = sqrt(r2);
            e += 0.5 * (Vr_d(r2, c) + si * sjv * Va_d(r, c));
            const double gg = dVr_over_r_d(r2, c) * r + si * sjv * dVa_d(r, c) +
                              (Ai + Aj) * domega_d(r, c.r_l, c.r_h);
            w += 0.5 * (-gg * r);
        });
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    sp[threadIdx.x] = pairs;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
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

constexpr int RED_TPB = 256;
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
// Caller order [n][3] doubles -> internal state in sorted order, and the
// fixed-point words.  FP32 mode: X = round(x 2^52 / L) (int64), V = two-float.
template <class M>
__global__ void __launch_bounds__(TPB) k_load_state(int n, Geom g, const double* __restrict__ pos_in,
                                                    const double* __restrict__ vel_in, const int* __restrict__ id,
                                                    void* __restrict__ xs, void* __restrict__ vs,
                                                    typename M::pos_t* __restrict__ pos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
    if constexpr (M::fp64) {
        double xx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xx[d] = pos_in[3 * (size_t)o + d];
            ((double*)xs)[(size_t)d * n + i] = xx[d];
            ((double*)vs)[(size_t)d * n + i] = vel_in ? vel_in[3 * (size_t)o + d] : 0.0;
        }
        pos[i] = ModeF64::from_x(xx[0], xx[1], xx[2], g);
    } else {
        int w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = pos_in[3 * (size_t)o + d];
            const long long P = __double2ll_rn(x * g.inv32[d] * 1048576.0);  // x 2^52 / L
            ((long long*)xs)[(size_t)d * n + i] = P;
            w[d] = ModeF32::word(P);
            const double v = vel_in ? vel_in[3 * (size_t)o + d] : 0.0;
            const float vh = (float)v;
            ((float2*)vs)[(size_t)d * n + i] = make_float2(vh, (float)(v - (double)vh));
        }
        pos[i] = make_int4(w[0], w[1], w[2], 0);
    }
}

template <class M>
__global__ void __launch_bounds__(TPB) k_store_state(int n, Geom g, const int* __restrict__ id,
                                                     const void* __restrict__ xs, const void* __restrict__ vs,
                                                     double* __restrict__ pos_out, double* __restrict__ vel_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x, v;
        if constexpr (M::fp64) {
            x = ((const double*)xs)[(size_t)d * n + i];
            v = ((const double*)vs)[(size_t)d * n + i];
        } else {
            x = (double)((const long long*)xs)[(size_t)d * n + i] * (g.s32d[d] * 9.5367431640625e-07);  // L / 2^52
            const float2 vv = ((const float2*)vs)[(size_t)d * n + i];
            v = (double)vv.x + (double)vv.y;
        }
        if (pos_out) pos_out[3 * (size_t)o + d] = x;
        if (vel_out) vel_out[3 * (size_t)o + d] = v;
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

// Lists in caller indices (diagnostics): staged index -> sorted index -> id.
__global__ void __launch_bounds__(TPB) k_store_nlist(int n, int cap_out, const int* __restrict__ id, ListRef L,
                                                     StageTable tb, int* __restrict__ nnb_out, int* __restrict__ nbr_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = i / TPB;
    const int R = tb.n[b];
    const int* off = tb.off + (size_t)b * (tb.cmax + 1);
    const int* base = tb.base + (size_t)b * tb.cmax;
    const int o = id[i];
    const int w = L.nnb[i];
    const int nn = w & 0xffff, nf = w >> 16;
    if (nnb_out) nnb_out[o] = nn + nf;
    if (!nbr_out) return;
    int k = 0;
    for_entries(L, n, i, nn, nf, [&](int s) {
        if (k >= cap_out) return;
        int lo = 0, hi = R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= s) lo = mid;
            else hi = mid - 1;
        }
        nbr_out[(size_t)o * cap_out + k++] = id[base[lo] + (s - off[lo])];
    });
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
