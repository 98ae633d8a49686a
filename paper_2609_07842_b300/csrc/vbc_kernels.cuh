// vbc_kernels.cuh -- CUDA kernels of the VBC path (sm_103a).
//
// Particles are stored sorted by cell, the cells ranked along a Morton curve.
// The cell grid (cells at least r_c + skin wide) is padded with empty
// phantom cells so that every aligned 4x2x2 group of cells holds consecutive
// ranks and its particles form one contiguous range of the sorted arrays.
// Every kernel that walks neighbour lists runs one thread block per group.
// The block first copies the 6x4x4 real cells around its group into shared
// memory (the staging), and the lists hold 16-bit indices into that staging,
// so a pass reads 2 bytes per list entry from HBM and serves every neighbour
// lookup from shared memory.
//
// One MD step:
//   rebuild (only when a particle moved more than skin/2 since the last build):
//     k_bin -> k_scan_sums -> k_scan_apply -> k_scatter -> k_cellsort ->
//     k_permute -> k_nlist (which also copies the gathered state back)
//   k_count   pass 1: n_i, s_i, s'_i                        (Eqs. counter, Psidelta)
//   k_chain   A_i = s'_i sum_j s_j V_a(r_ij), window particles only
//   k_force   pass 2: F_i, fused with the BAOAB update of the state
//   k_count_e, k_chain_e, k_energy   FP64 U, W and pair count (on request only)
// The rebuild kernels read a device flag and return at once when no rebuild
// is due, so the host never waits on the device between steps.  Every pass
// walks a full (both-direction) list and sums without floating-point
// atomics, so results do not depend on scheduling.
#pragma once

#include <climits>
#include <type_traits>

#include <cooperative_groups.h>

#include "vbc_device.cuh"

namespace vbc {

constexpr int TPB = 128;          // threads per block of the per-particle kernels
constexpr int SC_TPB = 128;       // threads per block of the cell-group kernels
constexpr int SCAN_CHUNK = 2048;  // cells per block in the two-pass scan
constexpr int SCAN_TPB = 256;
constexpr int MAX_CELL = 512;     // a denser cell means the system has collapsed

enum Epilogue { EPI_FORCE = 0, EPI_START = 1, EPI_FINISH = 2, EPI_FINISH_START = 3 };

// Waits until the preceding kernel of the stream has completed and its writes
// are visible.  A kernel launched with programmatic stream serialization may
// start before then (its launch overlaps the predecessor's last blocks); one
// launched plainly starts after it anyway, and the wait returns at once.
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Appends p to a work list whose length is *counter, with one atomic per set
// of lanes that append together (the counter is one word that every block
// of the grid appends to).  The order of a list is not part of any result:
// every listed particle is processed on its own.
__device__ __forceinline__ void list_append(int* __restrict__ list, int* counter, int p)
{
    const cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (int)g.size());
    base = g.shfl(base, 0);
    list[base + (int)g.thread_rank()] = p;
}

// ================================================================ rebuild: sort by cell
// The rebuild steps run only when a rebuild is due and nothing is halted.
__device__ __forceinline__ bool rebuild_on(const Status* st) { return st->rebuild && !st->frozen && !st->crowded; }

// Particle i of the cell binning (0 <= i < n): its cell's Morton rank and its
// slot in that cell; particle 0 also clears the build statistics.
template <class M>
__device__ __forceinline__ void bin_item(int i, const typename M::pos_t* __restrict__ pos, const Geom& g,
                                         const int* __restrict__ morton_rank, int* __restrict__ cell_of,
                                         int* __restrict__ slot_of, int* __restrict__ cell_count, Status* st)
{
    if (i == 0) {
        st->max_nnb = 0;
        st->nnb_sum = 0;
        st->max_stage = 0;
        st->max_own = 0;
    }
    const int3 c = cell_of_pos<M>(pos[i], g);
    const int key = morton_rank[(c.z * g.nc[1] + c.y) * g.nc[0] + c.x];
    cell_of[i] = key;
    slot_of[i] = atomicAdd(&cell_count[key], 1);
}

template <class M>
__global__ void __launch_bounds__(TPB) k_bin(const typename M::pos_t* __restrict__ pos, int n,
                                             Geom g, const int* __restrict__ morton_rank,
                                             int* __restrict__ cell_of, int* __restrict__ slot_of,
                                             int* __restrict__ cell_count, Status* st)
{
    if (!rebuild_on(st)) return;
    // as bin_item, with one atomic per cell and warp: particles arrive in the previous sorted
    // order, so neighbouring lanes mostly share a cell (the order within a cell is settled by
    // k_cellsort, whatever the slots)
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < n;
    int key = -1;
    if (act) {
        if (i == 0) {
            st->max_nnb = 0;
            st->nnb_sum = 0;
            st->max_stage = 0;
            st->max_own = 0;
        }
        const int3 c = cell_of_pos<M>(pos[i], g);
        key = morton_rank[(c.z * g.nc[1] + c.y) * g.nc[0] + c.x];
        cell_of[i] = key;
    }
    const unsigned active = __ballot_sync(0xffffffffu, act);
    if (!act) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned peers = __match_any_sync(active, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(&cell_count[key], __popc(peers));
    base = __shfl_sync(active, base, leader);
    slot_of[i] = base + __popc(peers & ((1u << lane) - 1u));
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
template <int NT>
__device__ __forceinline__ void scan_sums_chunk(int b, const int* __restrict__ cell_count, int ncell,
                                                int* __restrict__ chunk_sum, int* sw)
{
    const int base = b * SCAN_CHUNK;
    int s = 0;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += NT) {
        const int c = base + k;
        if (c < ncell) s += cell_count[c];
    }
    int total;
    block_exclusive_scan<NT>(s, sw, total);
    if (threadIdx.x == 0) chunk_sum[b] = total;
}

__global__ void __launch_bounds__(SCAN_TPB) k_scan_sums(const int* __restrict__ cell_count, int ncell,
                                                        int* __restrict__ chunk_sum, const Status* st)
{
    if (!rebuild_on(st)) return;
    __shared__ int sw[SCAN_TPB / 32];
    scan_sums_chunk<SCAN_TPB>(blockIdx.x, cell_count, ncell, chunk_sum, sw);
}

// Pass 2: chunk offset from the preceding chunk sums, then the local scan.
// Writes cell_start[0..ncell] and clears cell_count for the next build.
template <int NT>
__device__ __forceinline__ void scan_apply_chunk(int chunk, int* __restrict__ cell_count, int ncell,
                                                 const int* __restrict__ chunk_sum, int* __restrict__ cell_start,
                                                 Status* st, int* sw)
{
    int off = 0;
    for (int b = threadIdx.x; b < chunk; b += NT) off += chunk_sum[b];
    int tot;
    block_exclusive_scan<NT>(off, sw, tot);
    off = tot;  // sum over all preceding chunks
    constexpr int PER = SCAN_CHUNK / NT;
    const int base = chunk * SCAN_CHUNK + threadIdx.x * PER;
    int v[PER];
    int s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = (base + k < ncell) ? cell_count[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = off + block_exclusive_scan<NT>(s, sw, total);
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

__global__ void __launch_bounds__(SCAN_TPB) k_scan_apply(int* __restrict__ cell_count, int ncell,
                                                         const int* __restrict__ chunk_sum,
                                                         int* __restrict__ cell_start, Status* st)
{
    // raises `crowded` itself, so it does not test it
    if (!st->rebuild || st->frozen) return;
    __shared__ int sw[SCAN_TPB / 32];
    scan_apply_chunk<SCAN_TPB>(blockIdx.x, cell_count, ncell, chunk_sum, cell_start, st, sw);
}

__global__ void __launch_bounds__(TPB) k_scatter(int n, const int* __restrict__ cell_of,
                                                 const int* __restrict__ slot_of,
                                                 const int* __restrict__ cell_start,
                                                 int* __restrict__ order, const Status* st)
{
    if (!rebuild_on(st)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    order[cell_start[cell_of[i]] + slot_of[i]] = i;
}

// Window pairs of the FP32-split counts are measured finer than the 32-bit
// words.  A count error dn moves s'_i by s''_i dn, and A_i = s'_i sum_j s_j V_a
// multiplies that by the well sum, so a window particle of large A_i turns
// the ~1e-7 count error of the 32-bit position grid (L / 2^32 per axis) into
// a force error of order 1e-5 rms|F|.  The 64-bit state carries 20 more bits
// below each word; the top ten of them (P - word(P) 2^20, in [-2^19, 2^19),
// floored to a multiple of 2^10) are packed three to an int and added to the
// separation of window pairs only, which puts the count error near 1e-10.
// The packed ints sit in an array of their own beside the words, written
// wherever the state is (load, update, the rebuild's copy-back), so that a
// count reads one int per neighbour rather than three state words.
__device__ __forceinline__ int resid10(long long P)
{
    return (int)(((P + (1ll << 19)) & ((1ll << 20) - 1)) - (1ll << 19)) >> 10;
}
// Packed residuals of one particle from its coordinates (units L / 2^52).
__device__ __forceinline__ int pack_resid3(long long P0, long long P1, long long P2)
{
    return (resid10(P0) & 1023) | (resid10(P1) & 1023) << 10 | (resid10(P2) & 1023) << 20;
}
// Field k (0, 1, 2) of a packed residual, sign-extended.
__device__ __forceinline__ long long resid_field(int r, int k)
{
    return (long long)((int)((unsigned)r << (22 - 10 * k)) >> 22);
}
// Within each cell, order particles by their index in the previous sorted
// order, so that the layout (and every summation order) is a function of the
// previous layout and the positions only, not of atomic scheduling.  Cells of
// up to 16 particles are sorted in registers (odd-even transposition), larger
// ones by insertion in memory.
__device__ __forceinline__ void cellsort_item(int c, const int* __restrict__ cell_start, int* __restrict__ order)
{
    const int b = cell_start[c], e = cell_start[c + 1], cnt = e - b;
    if (cnt <= 1) return;
    if (cnt <= 16) {
        int v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = k < cnt ? order[b + k] : 0x7fffffff;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = r & 1; k + 1 < 16; k += 2) {
                const int lo = min(v[k], v[k + 1]), hi = max(v[k], v[k + 1]);
                v[k] = lo;
                v[k + 1] = hi;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < cnt) order[b + k] = v[k];
        return;
    }
    for (int k = b + 1; k < e; ++k) {
        const int o = order[k];
        int m = k - 1;
        while (m >= b && order[m] > o) {
            order[m + 1] = order[m];
            --m;
        }
        order[m + 1] = o;
    }
}

__global__ void __launch_bounds__(TPB) k_cellsort(int ncell, const int* __restrict__ cell_start,
                                                  int* __restrict__ order, const Status* st)
{
    if (!rebuild_on(st)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) cellsort_item(c, cell_start, order);
}

// Gathers the state (8-byte words: positions and velocities of either mode),
// the original index and the fixed-point position into sorted order.
template <class M>
__device__ __forceinline__ void permute_item(int k, int n, const int* __restrict__ order,
                                             const unsigned long long* __restrict__ x,
                                             const unsigned long long* __restrict__ v, const int* __restrict__ id,
                                             const typename M::pos_t* __restrict__ pos,
                                             unsigned long long* __restrict__ xt, unsigned long long* __restrict__ vt,
                                             int* __restrict__ idt, typename M::pos_t* __restrict__ post)
{
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
__device__ __forceinline__ void copyback_item(int k, int n, const unsigned long long* __restrict__ xt,
                                              const unsigned long long* __restrict__ vt, const int* __restrict__ idt,
                                              const typename M::pos_t* __restrict__ post,
                                              unsigned long long* __restrict__ x, unsigned long long* __restrict__ v,
                                              int* __restrict__ id, typename M::pos_t* __restrict__ pos,
                                              typename M::pos_t* __restrict__ xref, int* __restrict__ resid)
{
    unsigned long long xs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xs[a] = xt[(size_t)a * n + k];
        x[(size_t)a * n + k] = xs[a];
        v[(size_t)a * n + k] = vt[(size_t)a * n + k];
    }
    if constexpr (!M::fp64) resid[k] = pack_resid3((long long)xs[0], (long long)xs[1], (long long)xs[2]);
    id[k] = idt[k];
    const typename M::pos_t p = post[k];
    pos[k] = p;
    xref[k] = p;
}

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
    if (!rebuild_on(st)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) permute_item<M>(k, n, order, x, v, id, pos, xt, vt, idt, post);
}

// ================================================================ blocks of cells
// The cell grid is padded with empty phantom cells to extents that are
// multiples of (BXC, BYC, BZC), and cells are ranked along the Morton curve
// of the padded grid (code bits x0 y0 z0 x1 y1 z1 ... from the lowest).  An
// aligned BXC x BYC x BZC group of cells is then 2^BLOCK_BITS consecutive
// ranks, so its particles form one contiguous range of the sorted arrays.
// Every kernel that walks neighbour lists runs one thread block per such
// group.  The block first copies the (BXC+2) x (BYC+2) x (BZC+2) real cells
// around its group (periodic wrap on the real grid) into shared memory --
// the staging -- cell by cell in the order k = (lz SY + ly) SX + lx, so the
// three cells of one x row of a particle's 27-cell neighbourhood occupy one
// contiguous range of the staging.  List entries are 16-bit staging indices.
// The wrap needs at least 3 real cells per axis; with few cells a staged
// cell can appear twice, but the 27 cells around any one particle are
// distinct.
constexpr int BLOCK_BITS = 4;                    // Morton bits x0 y0 z0 x1
constexpr int BXC = 4, BYC = 2, BZC = 2;         // own cells per axis
constexpr int OWN_CELLS = BXC * BYC * BZC;       // 16
constexpr int SX = BXC + 2, SY = BYC + 2, SZ = BZC + 2;
constexpr int SCELLS = SX * SY * SZ;             // 96 staged cells
constexpr int SCELLS_P2 = 128;                   // offset table size (binary search)
static_assert(SCELLS <= SC_TPB && SCELLS <= SCELLS_P2, "one thread per staged cell");

struct SuperGrid {
    const int* morton_rank;  // real linear cell index -> rank on the padded Morton curve
    const int* sc_org;       // block -> coordinates of its first cell, x | y << 10 | z << 20
    const int* cell_start;   // rank -> sorted index of its first particle; [npad + 1]
};

// Per-block capacities (grown after an overflow).
struct SuperCaps {
    int smax;  // staged particles
    int omax;  // own particles (multiple of 32)
    int cap;   // list entries of one particle: the stride of the row slots (multiple of 8)
};

// Tables the list build leaves for the passes.
constexpr int CLOSE_K = 12;          // close entries kept per particle, as staging indices of its group
constexpr int CLOSE_NONE = 0xffff;   // an empty close-list slot
struct GroupAux {
    int* stage_idx;  // [groups][smax] sorted index of each staged particle
    int2* meta;      // [groups] (staged particles, own particles)
    int* grp;        // [n] cell group of each particle (whose staging its row's entries index)
    uint16_t* close; // [n][CLOSE_K] staging indices of close entries (near, then far within r_l), CLOSE_NONE for none
    void* fcore;     // [n] force and tag, float4 (FP32 mode) or F64x4 (w = 1: the particle's whole force)
    int* glist;      // [n] particles whose force the list-walking pass forms (k_count_near, k_chain)
};

struct SuperTab {
    int base[SCELLS];             // sorted index of each staged cell's first particle
    int off[SCELLS_P2 + 1];       // staging offset of each staged cell; total from SCELLS on
    int own[OWN_CELLS + 1];       // cell_start of the block's ranks
    int sw[SC_TPB / 32];          // scan scratch
};

// Reads the staging table of block s (whole block).  Returns the first own
// particle p0, the number of own particles and of staged particles.
__device__ __forceinline__ void load_group(int s, const Geom& g, const SuperGrid& G, SuperTab& T, int& p0,
                                               int& n_own, int& total)
{
    const int t = threadIdx.x;
    int cnt = 0;
    if (t < SCELLS) {
        const int org = __ldg(G.sc_org + s);
        int x = (org & 1023) - 1 + t % SX;
        int y = ((org >> 10) & 1023) - 1 + (t / SX) % SY;
        int z = (org >> 20) - 1 + t / (SX * SY);
        x = x < 0 ? x + g.nc[0] : (x >= g.nc[0] ? x - g.nc[0] : x);
        y = y < 0 ? y + g.nc[1] : (y >= g.nc[1] ? y - g.nc[1] : y);
        z = z < 0 ? z + g.nc[2] : (z >= g.nc[2] ? z - g.nc[2] : z);
        const int r = __ldg(G.morton_rank + (z * g.nc[1] + y) * g.nc[0] + x);
        const int b = __ldg(G.cell_start + r);
        cnt = __ldg(G.cell_start + r + 1) - b;
        T.base[t] = b;
    }
    if (t <= OWN_CELLS) T.own[t] = __ldg(G.cell_start + OWN_CELLS * s + t);
    int tot;
    const int o = block_exclusive_scan<SC_TPB>(cnt, T.sw, tot);
    if (t < SCELLS) T.off[t] = o;
    else if (t < SCELLS_P2) T.off[t] = tot;
    if (t == 0) T.off[SCELLS_P2] = tot;
    __syncthreads();
    p0 = T.own[0];
    n_own = T.own[OWN_CELLS] - p0;
    total = tot;
}

// Staged cell holding staging index m: the largest k with off[k] <= m.
__device__ __forceinline__ int staged_cell(const int* off, int m)
{
    int k = 0;
#pragma unroll
    for (int step = SCELLS_P2 / 2; step > 0; step >>= 1)
        if (off[k + step] <= m) k += step;
    return k;
}

// Sorted index of staging index m.
__device__ __forceinline__ int staged_index(const SuperTab& T, int m)
{
    const int k = staged_cell(T.off, m);
    return T.base[k] + (m - T.off[k]);
}

// Copies every staged particle: put(m, get(j)) for staging index m and
// sorted index j, B loads in flight per thread; with rec, also records j in
// rec[m] (the list build's staged-index table).
template <class V, int B = 4, class Get, class Put>
__device__ __forceinline__ void stage(const SuperTab& T, int total, Get&& get, Put&& put, int* rec = nullptr)
{
    for (int m0 = threadIdx.x; m0 < total; m0 += SC_TPB * B) {
        int jj[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int m = m0 + u * SC_TPB;
            jj[u] = m < total ? staged_index(T, m) : -1;
        }
        V v[B];
#pragma unroll
        for (int u = 0; u < B; ++u)
            if (jj[u] >= 0) v[u] = get(jj[u]);
#pragma unroll
        for (int u = 0; u < B; ++u)
            if (jj[u] >= 0) {
                put(m0 + u * SC_TPB, v[u]);
                if (rec) rec[m0 + u * SC_TPB] = jj[u];
            }
    }
}

// Own cell b (Morton low bits of its rank) of own particle p: the largest b
// with own[b] <= p.
__device__ __forceinline__ int own_cell(const SuperTab& T, int p)
{
    int b = 0;
#pragma unroll
    for (int step = OWN_CELLS / 2; step > 0; step >>= 1)
        if (T.own[b + step] <= p) b += step;
    return b;
}

// Staged cell number of own cell b (bits x0 y0 z0 x1).
__device__ __forceinline__ int own_staged_cell(int b)
{
    const int bx = (b & 1) | ((b >> 2) & 2), by = (b >> 1) & 1, bz = (b >> 2) & 1;
    return ((1 + bz) * SY + (1 + by)) * SX + (1 + bx);
}

// ---------------------------------------------------------------- lists
// The row of sorted particle p occupies the fixed slot nbr[p * cap ...]: its
// entries (staging indices of its cell group, grp[p]) in candidate order,
// padded to a multiple of 4 with the particle's own staging index, which adds
// exactly nothing to a force (d = 0).  nnb[p] = near | far << 16, near the
// entries closer than r_r + skin at the build, far the others up to r_c + skin.
__device__ __forceinline__ int pad4(int v) { return (v + 3) & ~3; }
__device__ __forceinline__ int row_len(int w) { return (w & 0xffff) + (w >> 16); }

// The 4 entries of one 8-byte chunk.
__device__ __forceinline__ void unpack4(const uint2 v, int h[4])
{
    h[0] = (int)(v.x & 0xffffu);
    h[1] = (int)(v.x >> 16);
    h[2] = (int)(v.y & 0xffffu);
    h[3] = (int)(v.y >> 16);
}

// Near (0), far (1) or beyond the list radius (-1).
struct ListParams {
    unsigned long long rlist2_fix, near2_fix, rl2_fix;
    double rlist2, near2, rl2;
    float rlist2_f, near2_f, rl2_f;  // float tests on block-relative coordinates (with a margin)
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
        const double r2 = __fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)));
        if (r2 >= lp.rlist2) return -1;
        return r2 < lp.near2 ? 0 : 1;
    }
};
// Float positions relative to the block's centre (FP32 mode, at least 8
// cells per axis so that the staging spans less than half the box): the
// classification only has to keep every pair within r_c + skin, so it tests
// against a radius enlarged by a relative 1e-5, far above the float error.
struct ListTestRel {
    __device__ __forceinline__ static int cls(const float4& a, const float4& b, const ListParams& lp)
    {
        const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
        if (r2 >= lp.rlist2_f) return -1;
        return r2 < lp.near2_f ? 0 : 1;
    }
};

// ---------------------------------------------------------------- shared-memory layouts
// Dynamic shared memory of each block kernel, carved in 16-byte aligned
// pieces; the host sizes its launches with the same functions.
__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

// The list build: the staged positions.
__host__ __device__ inline size_t nlist_smem(const SuperCaps& cp, size_t pos_bytes)
{
    return al16((size_t)cp.smax * pos_bytes);
}

// The energy kernels: staged positions and an optional staged value per particle.
struct PassLayout {
    size_t val, total;
};
__host__ __device__ inline PassLayout pass_layout(const SuperCaps& cp, size_t pos_bytes, size_t val_bytes)
{
    PassLayout l{};
    l.val = al16((size_t)cp.smax * pos_bytes);
    l.total = l.val + al16((size_t)cp.smax * val_bytes);
    return l;
}

// Shifts the 192-bit value (a2:a1:a0) right by s bits (left by -s when s < 0),
// |s| < 192; the close-list assembly of k_nlist.
__device__ __forceinline__ void shift192(unsigned long long& a0, unsigned long long& a1, unsigned long long& a2,
                                         int s)
{
    if (s >= 0) {
        while (s >= 64) {
            a0 = a1;
            a1 = a2;
            a2 = 0ull;
            s -= 64;
        }
        if (s) {
            a0 = (a0 >> s) | (a1 << (64 - s));
            a1 = (a1 >> s) | (a2 << (64 - s));
            a2 >>= s;
        }
    } else {
        s = -s;
        while (s >= 64) {
            a2 = a1;
            a1 = a0;
            a0 = 0ull;
            s -= 64;
        }
        if (s) {
            a2 = (a2 << s) | (a1 >> (64 - s));
            a1 = (a1 << s) | (a0 >> (64 - s));
            a0 <<= s;
        }
    }
}

// ================================================================ rebuild: lists
#ifndef NLIST_MIN_BLOCKS
#define NLIST_MIN_BLOCKS 8
#endif
// One block per cell group: stage the surrounding cells, then each thread
// takes own particles and scans the 9 contiguous x rows of their 27-cell
// neighbourhood, appending the accepted candidates (in candidate order) to
// the particle's fixed row slot nbr[p * cap ...].  The row is padded to a
// multiple of 4 entries with the particle's own staging index.
// The list build of cell group b (the whole block; smem is the dynamic shared
// memory of nlist_smem).  Raises `overflow` and `stage_overflow` itself.
// The copy-back of the sorted state, which the list build takes over from a
// pass of its own: the gathered state of the block's own particles moves
// from the sort's temporaries to the state arrays (copyback_item), while the
// build stages its neighbourhood from the temporaries.
template <class M>
struct CopyBack {
    int n;
    const unsigned long long *xt, *vt;
    const int* idt;
    const typename M::pos_t* post;
    unsigned long long *x, *v;
    int* id;
    typename M::pos_t *pos, *xref;
    int* resid;
};

template <class M>
__device__ __forceinline__ void copy_own(const CopyBack<M>* cb, int p0, int n_own)
{
    if (!cb) return;
    for (int j = threadIdx.x; j < n_own; j += SC_TPB)
        copyback_item<M>(p0 + j, cb->n, cb->xt, cb->vt, cb->idt, cb->post, cb->x, cb->v, cb->id, cb->pos, cb->xref,
                         cb->resid);
}

// With cb, pos is the sort's gathered positions (post) and the block also
// copies its own particles' state back (copy_own).
template <class M, bool REL>
__device__ __forceinline__ void nlist_group(int b, const Geom& g, const typename M::pos_t* __restrict__ pos,
                                            const SuperGrid& G, const SuperCaps& cp, const ListParams& lp,
                                            uint16_t* __restrict__ nbr, int* __restrict__ nnb, const GroupAux& aux,
                                            Status* st, unsigned char* smem, const CopyBack<M>* cb = nullptr)
{
    using pos_t = typename M::pos_t;
    using spos_t = typename std::conditional<REL, float4, pos_t>::type;
    __shared__ SuperTab T;
    __shared__ int s_mx;
    __shared__ unsigned long long s_sum;
    const int t = threadIdx.x;
    int p0, n_own, total;
    load_group(b, g, G, T, p0, n_own, total);
    if (t == 0) {
        atomicMax(&st->max_stage, total);
        atomicMax(&st->max_own, n_own);
        s_mx = 0;
        s_sum = 0;
        aux.meta[b] = make_int2(total, n_own);
    }
    if (total > cp.smax || n_own > cp.omax) {
        if (t == 0) {
            st->stage_overflow = 1;
            st->frozen_iter = (int)st->iter;
        }
        copy_own<M>(cb, p0, n_own);  // the state is complete even when the build is redone
        return;
    }
    spos_t* spos = (spos_t*)smem;
    int* sidx = aux.stage_idx + (size_t)b * cp.smax;  // the staged-index table the passes read
    if constexpr (REL) {
        // reference: the centre of the block's own cells (a cell boundary)
        const int org = __ldg(G.sc_org + b);
        const int cx[3] = {(org & 1023) + BXC / 2, ((org >> 10) & 1023) + BYC / 2, (org >> 20) + BZC / 2};
        uint32_t ref[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) ref[a] = (uint32_t)(((unsigned long long)cx[a] << 32) / (unsigned)g.nc[a]);
        stage<int4>(
            T, total, [&](int j) { return pos[j]; },
            [&](int m, const int4& v) {
                spos[m] = make_float4((float)(int)((uint32_t)v.x - ref[0]) * g.s32,
                                      (float)(int)((uint32_t)v.y - ref[1]) * g.s32,
                                      (float)(int)((uint32_t)v.z - ref[2]) * g.s32, 0.0f);
            },
            sidx);
    } else {
        stage<pos_t>(T, total, [&](int j) { return pos[j]; }, [&](int m, const pos_t& v) { spos[m] = v; }, sidx);
    }
    __syncthreads();
    int mx = 0;
    long long sum = 0;
    bool over = false;
    for (int j = t; j < n_own; j += SC_TPB) {
        const int p = p0 + j;
        const int ob = own_cell(T, p);
        const int kb = own_staged_cell(ob);
        const int mself = T.off[kb] + (p - T.own[ob]);
        const spos_t pi = spos[mself];
        uint16_t* row = nbr + (size_t)p * cp.cap;
        int len = 0, nn = 0;
        // close entries, as staging indices in registers until the end: up to CLOSE_K near
        // ones and, in scan order, up to CLOSE_K far ones within r_l (each shifted in from the
        // top of a 192-bit value)
        unsigned long long nw0 = 0ull, nw1 = 0ull, nw2 = 0ull;
        unsigned long long fw0 = 0ull, fw1 = 0ull, fw2 = 0ull;
        int nnc = 0, nfc = 0;
        unsigned long long buf = 0ull;  // up to 4 pending entries
#pragma unroll 1
        for (int d = 0; d < 9; ++d) {
            const int k0 = kb + (d / 3 - 1) * (SX * SY) + (d % 3 - 1) * SX - 1;
            const int e = T.off[k0 + 3];
            for (int base = T.off[k0]; base < e; base += 32) {
                // test up to 32 candidates into bit masks, then write the accepted ones.  Each
                // mask takes one bit per candidate, shifted in from the bottom, so candidate u
                // ends at bit cnt - 1 - u; in the FP32 mode the bit is the sign of r^2 minus
                // the threshold, moved in by a funnel shift (the sign of a float difference
                // is that of the exact one).
                const int cnt = min(32, e - base);
                uint32_t mnear = 0u, mlist = 0u, mrl = 0u;
#pragma unroll 4
                for (int u = 0; u < cnt; ++u) {
                    const int m = base + u;
                    if constexpr (REL) {
                        const float4 q = spos[m];
                        const float dx = pi.x - q.x, dy = pi.y - q.y, dz = pi.z - q.z;
                        const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
                        mnear = __funnelshift_l(__float_as_uint(r2 - lp.near2_f), mnear, 1);
                        mlist = __funnelshift_l(__float_as_uint(r2 - lp.rlist2_f), mlist, 1);
                        mrl = __funnelshift_l(__float_as_uint(r2 - lp.rl2_f), mrl, 1);
                    } else if constexpr (M::fp64) {
                        double dx, dy, dz;
                        ModeF64::delta64(pi, spos[m], g, dx, dy, dz);
                        const double r2 = __fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)));
                        mnear = (mnear << 1) | (r2 < lp.near2 ? 1u : 0u);
                        mlist = (mlist << 1) | (r2 < lp.rlist2 ? 1u : 0u);
                        mrl = (mrl << 1) | (r2 <= lp.rl2 ? 1u : 0u);
                    } else {
                        const int dx = pi.x - spos[m].x, dy = pi.y - spos[m].y, dz = pi.z - spos[m].z;
                        const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                                      (unsigned long long)((long long)dy * dy) +
                                                      (unsigned long long)((long long)dz * dz);
                        mnear = (mnear << 1) | (r2 < lp.near2_fix ? 1u : 0u);
                        mlist = (mlist << 1) | (r2 < lp.rlist2_fix ? 1u : 0u);
                        mrl = (mrl << 1) | (r2 <= lp.rl2_fix ? 1u : 0u);
                    }
                }
                // the particle itself (r = 0) is a candidate of its own cell
                if ((unsigned)(mself - base) < (unsigned)cnt) {
                    const uint32_t sb = ~(1u << (cnt - 1 - (mself - base)));
                    mnear &= sb;
                    mlist &= sb;
                }
                const int top = base + cnt - 1;  // the candidate at bit 0
                nn += __popc(mnear);
                // every accepted entry, in candidate order (highest bit first), four to an
                // 8-byte word of the row
                uint32_t ml = mlist;
                while (ml) {
                    const int hb = 31 - __clz(ml);
                    ml ^= 1u << hb;
                    buf = (buf >> 16) | ((unsigned long long)(top - hb) << 48);
                    if ((++len & 3) == 0 && len <= cp.cap)
                        *reinterpret_cast<unsigned long long*>(row + len - 4) = buf;
                }
                // close entries: the first CLOSE_K near ones, and far ones within r_l
                uint32_t mn = mnear;
                while (mn && nnc < CLOSE_K) {
                    const int hb = 31 - __clz(mn);
                    mn ^= 1u << hb;
                    shift192(nw0, nw1, nw2, 16);
                    nw2 |= (unsigned long long)(top - hb) << 48;
                    ++nnc;
                }
                uint32_t mfc = mlist & ~mnear & mrl;
                while (mfc && nfc < CLOSE_K) {
                    const int hb = 31 - __clz(mfc);
                    mfc ^= 1u << hb;
                    shift192(fw0, fw1, fw2, 16);
                    fw2 |= (unsigned long long)(top - hb) << 48;
                    ++nfc;
                }
            }
        }
        if (len <= cp.cap) {
            // the last 1..3 entries and the pads (the particle's own staging index)
            const int rem = len & 3;
            if (rem) {
                unsigned long long w = buf >> (16 * (4 - rem));
                for (int k = rem; k < 4; ++k) w |= (unsigned long long)mself << (16 * k);
                *reinterpret_cast<unsigned long long*>(row + (len & ~3)) = w;
            }
        }
        nnb[p] = nn | ((len - nn) << 16);
        aux.grp[p] = b;
        {
            // up to CLOSE_K close entries: the near entries, then far entries within r_l at the
            // build (for the per-particle count and soft-core force; a row with more near entries
            // than the list holds takes the list-walking force path).  Entry i of each kind sits at
            // bit 192 - 16 n + 16 i of its 192-bit value.
            const int kn = nnc;
            const int kf = min(nfc, CLOSE_K - kn);
            shift192(nw0, nw1, nw2, 16 * (CLOSE_K - kn));             // near entry i to slot i
            shift192(fw0, fw1, fw2, 16 * (CLOSE_K - nfc - kn));       // far entry i to slot kn + i (past 11: out)
            const int used = 16 * (kn + kf);
            unsigned long long m0 = ~0ull, m1 = ~0ull, m2 = ~0ull;  // ones over the empty slots
            shift192(m0, m1, m2, -used);
            uint2* cvo = reinterpret_cast<uint2*>(aux.close) + (CLOSE_K / 4) * (size_t)p;
            const unsigned long long w[3] = {nw0 | fw0 | m0, nw1 | fw1 | m1, nw2 | fw2 | m2};
#pragma unroll
            for (int k = 0; k < CLOSE_K / 4; ++k) cvo[k] = make_uint2((uint32_t)w[k], (uint32_t)(w[k] >> 32));
        }
        over |= len > cp.cap;
        mx = max(mx, len);
        sum += len;
    }
    copy_own<M>(cb, p0, n_own);
    // list statistics
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if ((t & 31) == 0) {
        atomicMax(&s_mx, mx);
        atomicAdd(&s_sum, (unsigned long long)sum);
    }
    const bool any_over = __syncthreads_or(over);
    if (t == 0) {
        atomicMax(&st->max_nnb, s_mx);
        atomicAdd((unsigned long long*)&st->nnb_sum, s_sum);
        if (b == 0) st->rebuilds += 1;
        if (any_over) {
            st->overflow = 1;
            st->frozen_iter = (int)st->iter;
        }
    }
}

// (The FP64 mode's wider positions take more registers: it asks for fewer resident blocks.)
template <class M, bool REL>
__global__ void __launch_bounds__(SC_TPB, M::fp64 ? NLIST_MIN_BLOCKS / 2 : NLIST_MIN_BLOCKS)
    k_nlist(Geom g, SuperGrid G, SuperCaps cp, ListParams lp, uint16_t* __restrict__ nbr, int* __restrict__ nnb,
            GroupAux aux, Status* st, CopyBack<M> cb)
{
    if (!rebuild_on(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    nlist_group<M, REL>(blockIdx.x, g, cb.post, G, cp, lp, nbr, nnb, aux, st, smem, &cb);
}

// ================================================================ pass 2: forces + BAOAB
struct StepArgs {
    void* x;              // [3][n] unwrapped positions (FP32 mode: int64 in units L / 2^52; FP64: double)
    void* v;              // [3][n] velocities (FP32 mode: int64 in units 2^-40; FP64: double)
    double* F_out;        // forces in caller order [n][3], or null (EPI_FORCE)
    // FP64 mode constants
    double dt, c1, c2;    // c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT)
    // FP32 mode constants (fixed point)
    float kick40;                        // (dt / 2) 2^40: force -> velocity units of a half kick
    float c2_40;                         // c2 2^40: normal -> velocity units
    unsigned long long dk_hi[3], dk_lo[3];  // (dt / 2) 2^12 / L_a: velocity units -> position units of a half drift
    unsigned long long c1_hi, c1_lo;        // c1 as integer part and 2^-64 fraction
    unsigned long long seed;
    float half_skin2;     // (skin / 2)^2
    int* resid;           // [n] packed residuals of the new positions (FP32 mode)
};

// State of one particle for its BAOAB update, loaded before the force loop
// so that the loads overlap it.
template <class M>
struct PState;
template <>
struct PState<ModeF32> {
    long long X[3];
    long long V[3];
    int4 xr;
    uint32_t id;
};
template <>
struct PState<ModeF64> {
    double X[3];
    double V[3];
    P64 xr;
    uint32_t id;
};

template <class M, int EPI>
__device__ __forceinline__ void load_pstate(int i, int n, const StepArgs& a, const int* __restrict__ id,
                                            const typename M::pos_t* __restrict__ xref, PState<M>& ps)
{
    constexpr bool start = EPI == EPI_START || EPI == EPI_FINISH_START;
    ps.id = (uint32_t)__ldg(id + i);
    if constexpr (EPI == EPI_FORCE) return;
    if constexpr (!M::fp64) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ps.V[d] = ((const long long*)a.v)[(size_t)d * n + i];
            if constexpr (start) ps.X[d] = ((const long long*)a.x)[(size_t)d * n + i];
        }
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ps.V[d] = ((const double*)a.v)[(size_t)d * n + i];
            ps.X[d] = ((const double*)a.x)[(size_t)d * n + i];
        }
    }
    if constexpr (start) ps.xr = xref[i];
}

// BAOAB update of particle i (unit mass, h = dt / 2) from its force.
// FP32 mode: positions are int64 in units of L / 2^52 and velocities int64
// in units of 2^-40, so the update needs no FP64 instruction: a kick adds
// the nearest integer of h F 2^40 (F from the FP32 force), a drift the exact
// fixed-point product v h 2^12 / L, and the friction a fixed-point product
// with c1.  FP64 mode: doubles.
template <class M, int EPI>
__device__ __forceinline__ void integrate(int i, int n, const Geom& g, typename M::real fx, typename M::real fy,
                                          typename M::real fz, const StepArgs& a, const PState<M>& ps, Status* st,
                                          typename M::pos_t* __restrict__ pos_next)
{
    constexpr bool start = EPI == EPI_START || EPI == EPI_FINISH_START;
    constexpr bool finish = EPI == EPI_FINISH || EPI == EPI_FINISH_START;
    bool bad = !isfinite(fx) || !isfinite(fy) || !isfinite(fz);
    if constexpr (!M::fp64) {
        long long* X = (long long*)a.x;
        long long* V = (long long*)a.v;
        const float f3[3] = {fx, fy, fz};
        float xi[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (start) {
            const float3 z = langevin_normals(a.seed, (unsigned long long)(st->step_base + st->iter), ps.id);
            xi[0] = z.x;
            xi[1] = z.y;
            xi[2] = z.z;
        }
        int w[3] = {0, 0, 0};
        int rp = 0;  // packed residuals of the new position
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            long long v = ps.V[d];
            const long long kick = float_to_ll_rn(f3[d] * a.kick40);
            if constexpr (finish) v += kick;                                       // B (closes the step)
            if constexpr (start) {
                long long P = ps.X[d];
                v += kick;                                                         // B
                P += mul_fix(v, a.dk_hi[d], a.dk_lo[d]);                           // A
                v = mul_fix(v, a.c1_hi, a.c1_lo) + float_to_ll_rn(a.c2_40 * xi[d]);  // O
                P += mul_fix(v, a.dk_hi[d], a.dk_lo[d]);                           // A
                X[(size_t)d * n + i] = P;
                w[d] = ModeF32::word(P);
                rp |= (resid10(P) & 1023) << (10 * d);
            }
            V[(size_t)d * n + i] = v;
        }
        if constexpr (start) {
            const int4 pn = make_int4(w[0], w[1], w[2], 0);
            pos_next[i] = pn;
            a.resid[i] = rp;
            const float ux = (float)(pn.x - ps.xr.x) * g.s32, uy = (float)(pn.y - ps.xr.y) * g.s32,
                        uz = (float)(pn.z - ps.xr.z) * g.s32;
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
            xs[d] = ps.X[d];
            vs[d] = ps.V[d];
        }
        // explicit fused multiply-adds: the rounding does not depend on the kernel this is inlined in
        if constexpr (finish) {
#pragma unroll
            for (int d = 0; d < 3; ++d) vs[d] = __fma_rn(h, f3[d], vs[d]);
        }
        if constexpr (start) {
            const double3 z = langevin_normals_d(a.seed, (unsigned long long)(st->step_base + st->iter), ps.id);
            const double zz[3] = {z.x, z.y, z.z};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                vs[d] = __fma_rn(h, f3[d], vs[d]);
                xs[d] = __fma_rn(h, vs[d], xs[d]);
                vs[d] = __fma_rn(a.c1, vs[d], __dmul_rn(a.c2, zz[d]));
                xs[d] = __fma_rn(h, vs[d], xs[d]);
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
            float d2 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float u = (float)(int)(ModeF64::hi32(pn, d) - ModeF64::hi32(ps.xr, d)) * (float)g.s32d[d];
                d2 += u * u;
            }
            if (d2 > a.half_skin2) st->rebuild = 1;
        }
    }
    if (bad) st->frozen = 1;
}
// Spare word of a staged position, holding s_j.
__device__ __forceinline__ void put_s(int4& p, float s) { p.w = __float_as_int(s); }
__device__ __forceinline__ void put_s(P64& p, double s) { p.w = (unsigned long long)__double_as_longlong(s); }
__device__ __forceinline__ float get_s(const int4& p) { return __int_as_float(p.w); }
__device__ __forceinline__ double get_s(const P64& p) { return __longlong_as_double((long long)p.w); }

// All terms of one pair in the FP32 mode, added to f (physical units).
__device__ __forceinline__ void pair_f32(const int4& pi, float si, float Ai, const int4& pj, float sj, float Aj,
                                         const Coef& c, const Geom& g, float& fx, float& fy, float& fz)
{
    const int ix = pi.x - pj.x, iy = pi.y - pj.y, iz = pi.z - pj.z;
    const unsigned long long r2i = (unsigned long long)((long long)ix * ix) +
                                   (unsigned long long)((long long)iy * iy) +
                                   (unsigned long long)((long long)iz * iz);
    const bool core = r2i < c.rr2_fix;
    const bool well = r2i > c.rr2_fix && r2i < c.ra2_fix && si * sj != 0.0f;
    const bool chain = r2i > c.rl2_fix && r2i < c.rh2_fix && Ai + Aj != 0.0f;
    if (!(core || well || chain)) return;
    // Every product and sum is spelt out (round-to-nearest intrinsics), so that no kernel
    // that inlines this contracts a multiply and an add differently from another: the
    // single-system walks and the batched launch give the same bits.
    const float dx = __fmul_rn((float)ix, g.s32), dy = __fmul_rn((float)iy, g.s32), dz = __fmul_rn((float)iz, g.s32);
    // the exact r^2 as one float (0.5 ulp): every term below starts from it, except the
    // well's r - r_m, which takes the exact integer difference (near the well's centre the
    // force is most sensitive to it)
    const float R = u64_to_float(r2i);
    const float r2 = __fmul_rn(R, g.s32sq);
    float gr = 0.0f;  // g / r
    if (core) gr = __fmul_rn(c.Er4f, __fmaf_rn(r2, c.rr2invf, -1.0f));
    if (well || chain) {
        float rinv = rsqrtf(r2);
        rinv = __fmul_rn(rinv, __fmaf_rn(__fmul_rn(__fmul_rn(-0.5f, r2), rinv), rinv, 1.5f));  // one Newton step
        const float r = __fmul_rn(r2, rinv);
        float gt = 0.0f;  // g from the well and the counts
        if (well) {
            const float u = __fdividef(__fmul_rn(s64_to_float((long long)r2i - (long long)c.rm2_fix), c.s2hinv),
                                       __fadd_rn(r, c.rmf));
            gt = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(si, sj), c.Ea4hf), u), __fmaf_rn(-u, u, 1.0f));
        }
        if (chain) {
            // (r - r_l) / w from r^2 - r_l^2 in fixed-point units (R and r_l^2 each within 0.5 ulp)
            const float tt = __fdividef(__fmul_rn(__fsub_rn(R, c.rl2_fixf), c.s2winv), __fadd_rn(r, c.rlf));
            const float h = __fmul_rn(__fmul_rn(__fmul_rn(__fadd_rn(Ai, Aj), 4.0f), tt), __fmaf_rn(-tt, tt, 1.0f));
            gt = __fmaf_rn(-h, c.winvf, gt);
        }
        gr = __fmaf_rn(gt, rinv, gr);
    }
    fx = __fmaf_rn(-gr, dx, fx);
    fy = __fmaf_rn(-gr, dy, fy);
    fz = __fmaf_rn(-gr, dz, fz);
}

// All terms of one pair in the FP64 mode.
__device__ __forceinline__ void pair_f64(const P64& pi, double si, double Ai, const P64& pj, double sj, double Aj,
                                         const Coef& c, const Geom& g, double& fx, double& fy, double& fz)
{
    double dx, dy, dz;
    ModeF64::delta64(pi, pj, g, dx, dy, dz);
    // explicit fused multiply-adds, as in r2_d: the same r^2 in every kernel this is inlined in
    const double r2 = __fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)));
    if (r2 >= c.rc2) return;
    const double r = sqrt(r2);
    double gr = dVr_over_r_d(r2, c);
    if (r > 0.0) gr += __fma_rn(Ai + Aj, domega_d(r, c.r_l, c.r_h), __dmul_rn(__dmul_rn(si, sj), dVa_d(r, c))) / r;
    fx = __fma_rn(-gr, dx, fx);
    fy = __fma_rn(-gr, dy, fy);
    fz = __fma_rn(-gr, dz, fz);
}


// ================================================================ pass 1: counts
// FP32-split: neighbours with r <= r_l add exactly 1 (an integer); window
// neighbours add omega in 2^-31 fixed point (window_weight_tab).  The
// threshold test t = n - (f - delta) is taken in the same fixed point, so
// s_i and s'_i carry only the error of the window terms, and the integer sums
// do not depend on the order of the terms.
// Saturation: when the close neighbours kept by the list build (up to
// CLOSE_K near entries) hold at least ceil(f - delta + 1) neighbours with r <= r_l, then
// n_i >= f - delta + 1 whatever the other entries add, so s_i = s'_i = 0
// exactly and nothing else is needed (unless the counts themselves are
// requested).  k_count_near tests that, one thread per particle, with direct
// loads of those few neighbours, and lists the particles it cannot settle;
// k_count_rows then walks their full rows, one warp per particle and one lane
// per entry, reading neighbours through the group's staged-index table.
// Both write s_i also into the spare word of the particle's position, where
// the force pass stages it.
struct CountOut {
    double* n_out;         // counts in caller order, or null
    long long* in_window;  // counter of window particles, or null
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
        // q = 1 - t^2 = (1 - t)(1 + t), with 1 - t taken from the exact fixed-point
        // difference: near the top of the window (t -> 1) the float 1 - t*t would lose
        // ~1e-6 of q to cancellation, and s' = -4 t q carries that into A_i
        const float t = (float)T * 4.656612873077393e-10f;                      // 2^-31
        const float omt = (float)(2147483648LL - T) * 4.656612873077393e-10f;  // 1 - t
        const float q = omt * (1.0f + t);
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

// r^2 of a window pair in units of (L / 2^32)^2 with the residuals ra, rb
// added: with d the word difference and e the residual difference (units of
// 2^-10 word), (d + e / 2^10)^2 = d^2 + 2 d e / 2^10 + e^2 / 2^20 per axis.
__device__ __forceinline__ unsigned long long r2_fine(const int4& a, int ra, const int4& b, int rb,
                                                      unsigned long long r2)
{
    const long long dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const long long ex = resid_field(ra, 0) - resid_field(rb, 0), ey = resid_field(ra, 1) - resid_field(rb, 1),
                    ez = resid_field(ra, 2) - resid_field(rb, 2);
    const long long cross = 2 * (dx * ex + dy * ey + dz * ez), sq = ex * ex + ey * ey + ez * ez;
    return (unsigned long long)((long long)r2 + ((cross + (sq >> 10)) >> 10));
}

// Squared separation for the FP64 paths.
template <class M>
__device__ __forceinline__ double r2_d(const typename M::pos_t& a, const typename M::pos_t& b, const Geom& g)
{
    double dx, dy, dz;
    M::delta64(a, b, g, dx, dy, dz);
    return __fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz)));
}

// s_i into the spare word of a position.
__device__ __forceinline__ void put_w(int4* p, float s) { reinterpret_cast<int*>(p)[3] = __float_as_int(s); }
__device__ __forceinline__ void put_w(P64* p, double s)
{
    reinterpret_cast<unsigned long long*>(p)[3] = (unsigned long long)__double_as_longlong(s);
}

// Force and tag of a particle: float4 in the FP32 mode, F64x4 in FP64.
struct __align__(32) F64x4 {
    double x, y, z, w;
};

// Index checks of the table-driven gathers.  The tables are consistent by
// construction (the list build writes them together and halts the system when
// a group outgrows its capacities); a check that fails anyway records the
// internal error in `bad` (reported by the host when the call ends) and the
// access is skipped, or redirected to particle 0, instead of leaving the
// buffers.
enum BadIndex { BAD_SORTED = 1, BAD_STAGED = 2, BAD_STAGING_SIZE = 3 };

__device__ __forceinline__ int checked_sorted(int jj, int n, int* bad)
{
    if ((unsigned)jj < (unsigned)n) return jj;
    *bad = BAD_SORTED;
    return 0;
}
__device__ __forceinline__ int checked_staged(int m, int cap, int* bad)
{
    if ((unsigned)m < (unsigned)cap) return m;
    *bad = BAD_STAGED;
    return 0;
}

// Copies a group's staged particles: put(m, j) for staging index m and sorted
// index j, four loads of the index table in flight per thread.  total is
// checked against the staging capacity cap and every j against n.
template <int NT = SC_TPB, class Put>
__device__ __forceinline__ void stage_by_table(const int* __restrict__ sidx, int total, int cap, int n, int* bad,
                                               Put&& put)
{
    constexpr int B = 4;
    if (total > cap) {
        *bad = BAD_STAGING_SIZE;
        total = cap;
    }
    for (int m0 = threadIdx.x; m0 < total; m0 += NT * B) {
        int jj[B];
#pragma unroll
        for (int u = 0; u < B; ++u) jj[u] = m0 + u * NT < total ? __ldg(sidx + m0 + u * NT) : -1;
#pragma unroll
        for (int u = 0; u < B; ++u)
            if (m0 + u * NT < total) {
                if ((unsigned)jj[u] < (unsigned)n) put(m0 + u * NT, jj[u]);
                else *bad = BAD_SORTED;
            }
    }
}

// k_count_near also forms, in the FP32 mode, the soft-core force of its
// particle from the same close neighbours.  Every pair inside the soft core
// is a near entry, so for a particle whose near entries all fit the close
// list the sum is its whole soft-core force; if the particle is saturated
// too (s_i = s'_i = 0, hence A_i = 0), it has no well term and its window
// terms need A_j != 0 of a neighbour -- which k_chain rules out by clearing
// the tag of every list neighbour of a window particle.  Every other particle
// goes on the list of k_force_rows.

// What the close count of own particle p reads besides the staging: its
// position, its close entries and its near-entry count (loaded ahead of the
// staging, so that the loads overlap).
template <class M>
struct NearOwn {
    typename M::pos_t pi;
    uint2 cv[CLOSE_K / 4];
    int nn;
};

template <class M>
__device__ __forceinline__ void load_near_own(int p, const typename M::pos_t* __restrict__ pos, const GroupAux& aux,
                                              const int* __restrict__ nnb, NearOwn<M>& o)
{
    o.nn = __ldg(nnb + p) & 0xffff;
    o.pi = pos[p];
    const uint2* cv = reinterpret_cast<const uint2*>(aux.close) + (CLOSE_K / 4) * (size_t)p;
#pragma unroll
    for (int k = 0; k < CLOSE_K / 4; ++k) o.cv[k] = __ldg(cv + k);
}

// The close count of own particle p from its close entries (staged positions
// in spos), with its outputs: s_i = s'_i = 0 and, in the FP32 mode, the
// soft-core force with the whole-force tag for a saturated particle; the
// work lists of the row walks for every other one.  With out.n_out (FP64
// counts wanted) no particle is settled here.
template <class M>
__device__ __forceinline__ void count_near_particle(int p, const NearOwn<M>& o, const typename M::pos_t* spos,
                                                    int total, const Geom& g, const Coef& c, typename M::pos_t* __restrict__ pos,
                                                    const GroupAux& aux, typename M::real* __restrict__ ds_out,
                                                    typename M::real2* __restrict__ sA, const CountOut& out,
                                                    int* __restrict__ ulist, Status* st)
{
    using pos_t = typename M::pos_t;
    using real = typename M::real;
    using real2 = typename M::real2;
    int full = 0;
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    if (!out.n_out) {
        int q[CLOSE_K];
#pragma unroll
        for (int k = 0; k < CLOSE_K / 4; ++k) unpack4(o.cv[k], q + 4 * k);
        // soft core: g / r = K (r^2 - r_r^2), r^2 in units of (L / 2^32)^2
        const float kc = c.Er4f * c.rr2invf * g.s32sq;
#pragma unroll
        for (int k = 0; k < CLOSE_K; ++k) {
            if (q[k] == CLOSE_NONE) continue;
            const pos_t pj = spos[checked_staged(q[k], total, &st->bad_index)];
            if constexpr (M::fp64) {
                full += r2_d<M>(o.pi, pj, g) <= c.rl2;
            } else {
                const unsigned long long r2i = r2_fix(o.pi, pj);
                full += r2i <= c.rl2_fix;
                if (r2i < c.rr2_fix) {
                    const float dx = (float)(o.pi.x - pj.x), dy = (float)(o.pi.y - pj.y), dz = (float)(o.pi.z - pj.z);
                    const float gr = __fmaf_rn(kc, __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz)), -c.Er4f);
                    fx = __fmaf_rn(-gr, dx, fx);
                    fy = __fmaf_rn(-gr, dy, fy);
                    fz = __fmaf_rn(-gr, dz, fz);
                }
            }
        }
    }
    const bool sat = !out.n_out && full >= c.sat_full;
    if (sat) {
        ds_out[p] = (real)0;
        sA[p] = real2{(real)0, (real)0};
        put_w(pos + p, (real)0);
    } else {
        ds_out[p] = (real)NAN;  // marks the particle for k_count_rows
        ulist[atomicAdd(&st->nu, 1)] = p;
    }
    const bool whole = !M::fp64 && sat && o.nn <= CLOSE_K;
    if constexpr (M::fp64) {
        static_cast<F64x4*>(aux.fcore)[p] = F64x4{0.0, 0.0, 0.0, 0.0};
    } else {
        static_cast<float4*>(aux.fcore)[p] = make_float4(fx * g.s32, fy * g.s32, fz * g.s32, whole ? 1.0f : 0.0f);
    }
    if (!whole) aux.glist[atomicAdd(&st->ngen, 1)] = p;
}

// The close count of cell group b (the whole block; smem holds the group's
// staged positions).  Starts with a block barrier, so that it may follow
// another group's work on the same shared memory.  (The fused batch launch;
// k_count_near runs the same per-particle count with its loads pipelined.)
template <class M>
__device__ __forceinline__ void count_near_group(int b, int n, const Geom& g, const Coef& c,
                                                 typename M::pos_t* __restrict__ pos, const SuperGrid& G,
                                                 const SuperCaps& cp, const GroupAux& aux,
                                                 const int* __restrict__ nnb, typename M::real* __restrict__ ds_out,
                                                 typename M::real2* __restrict__ sA, const CountOut& out,
                                                 int* __restrict__ ulist, Status* st, unsigned char* smem)
{
    using pos_t = typename M::pos_t;
    pos_t* spos = (pos_t*)smem;
    __syncthreads();  // the previous group is done with the shared positions
    const int p0 = __ldg(G.cell_start + OWN_CELLS * b);
    const int n_own = __ldg(G.cell_start + OWN_CELLS * b + OWN_CELLS) - p0;
    const int total = min(__ldg(aux.meta + b).x, cp.smax);
    if (!out.n_out)
        stage_by_table(aux.stage_idx + (size_t)b * cp.smax, __ldg(aux.meta + b).x, cp.smax, n, &st->bad_index,
                       [&](int m, int jj) { spos[m] = pos[jj]; });
    __syncthreads();
    for (int j = threadIdx.x; j < n_own; j += SC_TPB) {
        NearOwn<M> o;
        load_near_own<M>(p0 + j, pos, aux, nnb, o);
        count_near_particle<M>(p0 + j, o, spos, total, g, c, pos, aux, ds_out, sA, out, ulist, st);
    }
}

// Asynchronous 16-byte copy from global to shared memory (cp.async, bypassing
// L1), and the wait for every copy this thread issued.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Staged particles per thread whose table entries k_count_near loads one
// group ahead (the staging of a group holds about 680 particles at
// rho = 0.5; slots past NEAR_B * SC_TPB are copied synchronously).
constexpr int NEAR_B = 8;

// Range and staged total of cell group b.
struct GroupRange {
    int p0, n_own, total;
};
__device__ __forceinline__ GroupRange group_range(int b, const SuperGrid& G, const GroupAux& aux)
{
    GroupRange r;
    r.p0 = __ldg(G.cell_start + OWN_CELLS * b);
    r.n_own = __ldg(G.cell_start + OWN_CELLS * b + OWN_CELLS) - r.p0;
    r.total = __ldg(aux.meta + b).x;
    return r;
}

// k_count_near: the cell groups on a resident grid, each block taking groups
// b, b + gridDim.x, ...  The loads are pipelined so that each group waits on
// one memory round trip: the range of the group after next and the
// staged-index table of the next group are loaded while the current group
// is counted, and the staging copies (cp.async) overlap the loads of the own
// particles' close entries.
template <class M>
__global__ void __launch_bounds__(SC_TPB) k_count_near(int ngroups, int n, Geom g, Coef c,
                                                       typename M::pos_t* __restrict__ pos,
                                                       SuperGrid G, SuperCaps cp, GroupAux aux,
                                                       const int* __restrict__ nnb, typename M::real* __restrict__ ds_out,
                                                       typename M::real2* __restrict__ sA, CountOut out,
                                                       int* __restrict__ ulist, Status* st, int gated)
{
    // The launch beside a graph iteration's conditional returns when the iteration rebuilds
    // (the conditional's body then counts).  It decides from the flags the previous update
    // left: the rebuild flag is cleared only by k_count_rows, which waits for both counts,
    // and a halt the rebuild raises meanwhile makes every block return below as well.
    if (gated && st->rebuild && !halted(st)) return;
    using pos_t = typename M::pos_t;
    if (halted(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    if (out.n_out) {
        // FP64 counts wanted: no particle is settled here, nothing is staged
        for (int b = blockIdx.x; b < ngroups; b += gridDim.x)
            count_near_group<M>(b, n, g, c, pos, G, cp, aux, nnb, ds_out, sA, out, ulist, st, smem);
        return;
    }
    pos_t* spos = (pos_t*)smem;
    constexpr int CHUNKS = (int)(sizeof(pos_t) / 16);
    const int t = threadIdx.x;
    int b = blockIdx.x;
    if (b >= ngroups) return;
    GroupRange cur = group_range(b, G, aux);
    GroupRange nxt{0, 0, 0};
    if (b + (int)gridDim.x < ngroups) nxt = group_range(b + gridDim.x, G, aux);
    int* bad = &st->bad_index;
    int jj[NEAR_B];
    {
        const int* sidx = aux.stage_idx + (size_t)b * cp.smax;
        if (cur.total > cp.smax) {
            *bad = BAD_STAGING_SIZE;
            cur.total = cp.smax;
        }
#pragma unroll
        for (int u = 0; u < NEAR_B; ++u) jj[u] = t + u * SC_TPB < cur.total ? __ldg(sidx + t + u * SC_TPB) : -1;
    }
    for (; b < ngroups; b += gridDim.x) {
        __syncthreads();  // the previous group is done with the shared positions
        // this group's staging: asynchronous copies, then the rest (if any) synchronously
#pragma unroll
        for (int u = 0; u < NEAR_B; ++u)
            if (t + u * SC_TPB < cur.total) {
                const int j = checked_sorted(jj[u], n, bad);
#pragma unroll
                for (int k = 0; k < CHUNKS; ++k)
                    cp_async16(reinterpret_cast<int4*>(spos + t + u * SC_TPB) + k,
                               reinterpret_cast<const int4*>(pos + j) + k);
            }
        const int* sidx = aux.stage_idx + (size_t)b * cp.smax;
        for (int m = t + NEAR_B * SC_TPB; m < cur.total; m += SC_TPB) spos[m] = pos[checked_sorted(__ldg(sidx + m), n, bad)];
        // the first own particle of this thread
        NearOwn<M> o;
        const bool own0 = t < cur.n_own;
        if (own0) load_near_own<M>(cur.p0 + t, pos, aux, nnb, o);
        // the next group's table and the range of the one after it
        const int bn = b + gridDim.x;
        GroupRange nn2{0, 0, 0};
        if (bn < ngroups) {
            const int* sn = aux.stage_idx + (size_t)bn * cp.smax;
#pragma unroll
            for (int u = 0; u < NEAR_B; ++u) jj[u] = t + u * SC_TPB < nxt.total ? __ldg(sn + t + u * SC_TPB) : -1;
            if (bn + (int)gridDim.x < ngroups) nn2 = group_range(bn + gridDim.x, G, aux);
        }
        if (nxt.total > cp.smax) {
            *bad = BAD_STAGING_SIZE;
            nxt.total = cp.smax;
        }
        cp_async_wait_all();
        __syncthreads();
        if (own0) count_near_particle<M>(cur.p0 + t, o, spos, cur.total, g, c, pos, aux, ds_out, sA, out, ulist, st);
        for (int j = t + SC_TPB; j < cur.n_own; j += SC_TPB) {
            load_near_own<M>(cur.p0 + j, pos, aux, nnb, o);
            count_near_particle<M>(cur.p0 + j, o, spos, cur.total, g, c, pos, aux, ds_out, sA, out, ulist, st);
        }
        cur = nxt;
        nxt = nn2;
    }
}

// ================================================================ row walks
// k_count_rows, k_chain and k_force_rows walk the full list rows of the
// particles on their work lists.  Each picks its mode on the device from the
// list length.  Sparse, while the list holds at most n / DENSE_DIV particles:
// one warp per listed particle, one lane per entry, neighbours read through
// the group's staged-index table.  Dense otherwise: one block per cell group,
// which stages its neighbourhood in shared memory; a lane group of tpp
// threads walks each listed own particle's row, tpp the largest power of two
// (at most tmax <= 32) with (listed particles) * tpp <= NT, each thread
// taking every tpp-th 4-entry chunk.  NT (threads per block: 128, 256 or 512)
// and tmax are grid settings (vbc_set_tuning).  The order of the terms
// depends only on the row, the mode and these settings, so every result is a
// function of the state and the settings alone; the integer counts do not
// depend on the settings at all.  Both modes run a grid that stays resident
// (a few blocks per SM), the dense one taking the cell groups in a
// grid-stride loop.
constexpr int DENSE_DIV = 16;

template <int NT>
__device__ __forceinline__ int dense_tpp(int nl, int tmax)
{
    int t = tmax;
    while (t > 1 && nl * t > NT) t >>= 1;
    return t;
}

// The sparse walk of particle p's row with the lane's first entry loaded up
// front, beside the row length and the group index rather than after them
// (one dependent round trip less per listed particle).  Every lane below cap
// reads inside the particle's row slot; entries at or past len are not used.
struct LaneRow {
    const uint16_t* row;
    int h0;
};
__device__ __forceinline__ LaneRow lane_row(const uint16_t* __restrict__ nbr, int p, int cap)
{
    const uint16_t* row = nbr + (size_t)p * cap;
    const int lane = threadIdx.x & 31;
    return LaneRow{row, lane < cap ? (int)__ldg(row + lane) : 0};
}
template <class Visit>
__device__ __forceinline__ void walk_lanes_from(const LaneRow& r, int len, Visit&& visit)
{
    const int lane = threadIdx.x & 31;
    if (lane < len) visit(r.h0);
    for (int e = lane + 32; e < len; e += 32) visit((int)__ldg(r.row + e));
}

// Dense walk: 4-entry chunk k on thread k mod tpp of the lane group.  Rows
// start on 4-entry boundaries; the pads after the last entry are skipped.
template <class Visit>
__device__ __forceinline__ void walk_chunks(const uint16_t* __restrict__ row, int len, int sub, int tpp, Visit&& visit)
{
    for (int e0 = 4 * sub; e0 < len; e0 += 4 * tpp) {
        int h[4];
        unpack4(__ldg(reinterpret_cast<const uint2*>(row + e0)), h);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (e0 + k < len) visit(h[k]);
    }
}

// The same with the pads visited too: a pad repeats the particle's own
// staging index (separation 0), which adds exactly nothing to a force sum,
// so the force walk needs no test per entry.
template <class Visit>
__device__ __forceinline__ void walk_chunks_padded(const uint16_t* __restrict__ row, int len, int sub, int tpp,
                                                   Visit&& visit)
{
    for (int e0 = 4 * sub; e0 < len; e0 += 4 * tpp) {
        int h[4];
        unpack4(__ldg(reinterpret_cast<const uint2*>(row + e0)), h);
#pragma unroll
        for (int k = 0; k < 4; ++k) visit(h[k]);
    }
}

// Sum over an aligned lane group of w lanes (a power of two); every lane of
// the warp takes part.
template <class T>
__device__ __forceinline__ T group_sum(T v, int w)
{
    for (int o = w >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared memory of a dense row walk: staged positions, one extra value per
// staged particle, and a list of own particles.
struct DenseLayout {
    size_t extra, plist, total;
};
__host__ __device__ inline DenseLayout dense_layout(const SuperCaps& cp, size_t pos_bytes, size_t extra_bytes)
{
    DenseLayout l{};
    l.extra = al16((size_t)cp.smax * pos_bytes);
    l.plist = l.extra + al16((size_t)cp.smax * extra_bytes);
    l.total = l.plist + al16((size_t)cp.omax * 4);
    return l;
}

// Shared memory of the chunk-parallel dense count (FP32 split): staged
// positions, the list of own particles, each listed row's first chunk
// (exclusive scan, one extra slot for the total) and its fixed-point sum.
struct CountLayout {
    size_t plist, cstart, acc, total;
};
__host__ __device__ inline CountLayout count_layout(const SuperCaps& cp, size_t pos_bytes)
{
    CountLayout l{};
    l.plist = al16((size_t)cp.smax * pos_bytes);
    l.cstart = l.plist + al16((size_t)cp.omax * 4);
    l.acc = l.cstart + al16((size_t)(cp.omax + 1) * 4);
    l.total = l.acc + (size_t)cp.omax * 8;
    return l;
}


// Lists the own particles of group b that pick(j) selects (j from 0), at
// most cap of them (the list's capacity; more is an internal error recorded
// in bad); the whole block calls it.  Returns their number.
template <int NT, class Pick>
__device__ __forceinline__ int list_own(int n_own, int* plist, int* s_n, int cap, int* bad, Pick&& pick)
{
    if (threadIdx.x == 0) *s_n = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < n_own; j += NT)
        if (pick(j)) {
            const int k = atomicAdd(s_n, 1);
            if (k < cap) plist[k] = j;
            else *bad = BAD_STAGING_SIZE;
        }
    __syncthreads();
    return min(*s_n, cap);
}

// Runs body(u, sub, tpp) for the listed particles of a dense walk: slot u of
// the list (u >= nl on idle lanes, which must still take part in the lane
// group's sums), thread sub of its lane group.
template <int NT, class Body>
__device__ __forceinline__ void dense_rounds(int nl, int tmax, Body&& body)
{
    const int tpp = dense_tpp<NT>(nl, tmax), per_warp = 32 / tpp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = warp * per_warp; base < nl; base += (NT / 32) * per_warp)
        body(base + lane / tpp, lane & (tpp - 1), tpp);
}

// Count of one row over a lane group of `width` lanes, the result on every
// lane of it: s_i, s'_i and (if wanted) n_i.  walk(visit) calls visit(m)
// for this lane's entries.
// In the FP32 mode ri is the packed residual of i and resid(m) that of entry m
// (unused in FP64).
template <class M, class Walk, class Fetch, class Resid>
__device__ __forceinline__ void count_row(const typename M::pos_t& pi, int ri, Walk&& walk, int width, Fetch&& fetch,
                                          Resid&& resid, const Coef& c, const Geom& g, bool want_n,
                                          typename M::real& s, typename M::real& ds, double& n_val)
{
    if constexpr (M::fp64) {
        double acc = 0.0;
        walk([&](int m) {
            const double r2 = r2_d<M>(pi, fetch(m), g);
            if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
        });
        acc = group_sum(acc, width);
        s = omega_d(acc, c.fd, c.fd + 1.0);
        ds = domega_d(acc, c.fd, c.fd + 1.0);
        n_val = acc;
    } else {
        int full = 0;  // a row holds at most MAX_CAP (4096) entries
        unsigned long long q = 0;
        walk([&](int m) {
            const typename M::pos_t pj = fetch(m);
            const unsigned long long r2 = r2_fix(pi, pj);
            if (r2 < c.rh2_fix) {
                if (r2 <= c.rl2_fix) {
                    ++full;
                } else {
                    // omega has zero slope at both ends of the window, so a pair that the
                    // finer separation moves across r_l or r_h changes n_i by O(dr^2)
                    const unsigned long long rf = r2_fine(pi, ri, pj, resid(m), r2);
                    if (rf <= c.rl2_fix) q += 2147483648ull;
                    else if (rf < c.rh2_fix) q += window_weight_tab(rf - c.rl2_fix, c.wtab, c.wsh);
                }
            }
        });
        full = group_sum(full, width);
        q = group_sum(q, width);
        const long long Tf = ((long long)full << 31) + (long long)q - c.fd_fix;
        switch_from_fix(Tf, s, ds);
        n_val = 0.0;
        if (want_n) n_val = (double)full + (double)q * 4.656612873077393e-10;
    }
}

// Results of one counted row (one lane of the group).
template <class M>
__device__ __forceinline__ void count_row_out(int p, typename M::real s, typename M::real ds, double n_val,
                                              typename M::pos_t* __restrict__ pos, typename M::real* __restrict__ ds_out,
                                              typename M::real2* __restrict__ sA, const int* __restrict__ id,
                                              const CountOut& out, int* __restrict__ wpart, Status* st)
{
    using real = typename M::real;
    using real2 = typename M::real2;
    ds_out[p] = ds;
    sA[p] = real2{s, (real)0};
    put_w(pos + p, s);
    if (out.n_out) out.n_out[id[p]] = n_val;
    if (ds != (real)0) {
        // the chain-rule pass visits the window particles listed here
        list_append(wpart, &st->nwin, p);
        if (out.in_window) atomicAdd((unsigned long long*)out.in_window, 1ull);
    }
}

// Everything a row walk reads and writes (all three walks).
template <class M>
struct RowArgs {
    int n;
    Geom g;
    Coef c;
    typename M::pos_t* pos;
    SuperGrid G;
    SuperCaps cp;
    GroupAux aux;
    const uint16_t* nbr;
    const int* nnb;
    const int* id;
    typename M::real* ds;
    typename M::real2* sA;
    CountOut out;
    int* ulist;
    int* wpart;
    const int* resid;    // [n] packed residuals of the positions (FP32 mode)
    Status* st;
};

// Packed residuals of sorted particle j (FP32 mode; X is the state [3][n]); an
// index outside [0, n) is refused and reported rather than read.
template <class M>
__device__ __forceinline__ int resid_of(const RowArgs<M>& A, int j)
{
    if (M::fp64) return 0;
    if ((unsigned)j >= (unsigned)A.n) {
        A.st->bad_index = 1;
        return 0;
    }
    return __ldg(A.resid + j);
}

// Sorted index of row entry m of a particle of the group whose staged-index
// table is sidx (sparse walks), both indices checked.
template <class M>
__device__ __forceinline__ int table_index(const RowArgs<M>& A, const int* sidx, int m)
{
    return checked_sorted(__ldg(sidx + checked_staged(m, A.cp.smax, &A.st->bad_index)), A.n, &A.st->bad_index);
}

// Sparse count: list entry k of the particles k_count_near could not settle
// (one warp, one lane per row entry).
template <class M>
__device__ __forceinline__ void count_rows_item(const RowArgs<M>& A, int k)
{
    using real = typename M::real;
    const int p = A.ulist[k];
    const LaneRow lr = lane_row(A.nbr, p, A.cp.cap);
    const int b = __ldg(A.aux.grp + p);
    const int* sidx = A.aux.stage_idx + (size_t)b * A.cp.smax;
    const int len = row_len(__ldg(A.nnb + p));
    real s, ds;
    double n_val;
    count_row<M>(A.pos[p], resid_of(A, p), [&](auto&& v) { walk_lanes_from(lr, len, v); }, 32,
                 [&](int m) { return A.pos[table_index(A, sidx, m)]; },
                 [&](int m) { return resid_of(A, table_index(A, sidx, m)); }, A.c, A.g, A.out.n_out != nullptr, s, ds,
                 n_val);
    if ((threadIdx.x & 31) == 0) count_row_out<M>(p, s, ds, n_val, A.pos, A.ds, A.sA, A.id, A.out, A.wpart, A.st);
}

// Dense count of cell group b: the own particles that k_count_near marked
// (s'_i = NaN), the group's neighbourhood staged in smem (whole block;
// starts with a block barrier).
template <int NT>
__device__ void count_rows_group_chunks(const RowArgs<ModeF32>& A, int b, unsigned char* smem, int* s_n);

template <class M, int NT>
__device__ __forceinline__ void count_rows_group(const RowArgs<M>& A, int b, int tmax, unsigned char* smem, int* s_n)
{
    using pos_t = typename M::pos_t;
    using real = typename M::real;
    if constexpr (!M::fp64) {
        count_rows_group_chunks<NT>(A, b, smem, s_n);
        return;
    }
    const DenseLayout ly = dense_layout(A.cp, sizeof(pos_t), 0);
    pos_t* spos = (pos_t*)smem;
    int* plist = (int*)(smem + ly.plist);
    __syncthreads();  // the previous group is done with the shared arrays
    const int p0 = __ldg(A.G.cell_start + OWN_CELLS * b);
    const int n_own = __ldg(A.G.cell_start + OWN_CELLS * b + OWN_CELLS) - p0;
    const int nl = list_own<NT>(n_own, plist, s_n, A.cp.omax, &A.st->bad_index,
                                [&](int j) { return isnan(A.ds[p0 + j]); });
    if (nl == 0) return;
    // the count reads no s_j, so the spare word of a staged position holds its residuals
    stage_by_table<NT>(A.aux.stage_idx + (size_t)b * A.cp.smax, __ldg(A.aux.meta + b).x, A.cp.smax, A.n,
                       &A.st->bad_index, [&](int m, int jj) {
                           pos_t pj = A.pos[jj];
                           if constexpr (!M::fp64) pj.w = resid_of(A, jj);
                           spos[m] = pj;
                       });
    __syncthreads();
    dense_rounds<NT>(nl, tmax, [&](int u, int sub, int tpp) {
        const bool act = u < nl;
        const int p = p0 + (act ? plist[u] : 0);
        const uint16_t* row = A.nbr + (size_t)p * A.cp.cap;
        const int len = act ? row_len(__ldg(A.nnb + p)) : 0;
        real s, ds;
        double n_val;
        count_row<M>(A.pos[p], act ? resid_of(A, p) : 0, [&](auto&& v) { walk_chunks(row, len, sub, tpp, v); }, tpp,
                     [&](int m) { return spos[checked_staged(m, A.cp.smax, &A.st->bad_index)]; },
                     [&](int m) { return (int)spos[checked_staged(m, A.cp.smax, &A.st->bad_index)].w; }, A.c, A.g,
                     A.out.n_out != nullptr, s, ds, n_val);
        if (act && sub == 0) count_row_out<M>(p, s, ds, n_val, A.pos, A.ds, A.sA, A.id, A.out, A.wpart, A.st);
    });
}

// s_i, s'_i (and n_i) of sorted particle p from its fixed-point count acc
// = n_i 2^31 (the FP32 split's integer count and window weights, exact),
// then the outputs of a counted row.
__device__ __forceinline__ void finish_count_fix(const RowArgs<ModeF32>& A, int p, unsigned long long acc)
{
    const long long Tf = (long long)acc - A.c.fd_fix;
    float s, ds;
    switch_from_fix(Tf, s, ds);
    const double n_val = A.out.n_out ? (double)acc * 4.656612873077393e-10 : 0.0;  // exact: acc < 2^53
    count_row_out<ModeF32>(p, s, ds, n_val, A.pos, A.ds, A.sA, A.id, A.out, A.wpart, A.st);
}

// Dense count of cell group b, FP32 split, parallel over the 4-entry chunks
// of the listed rows rather than over rows: the rows of the group's
// unsettled own particles are laid end to end in chunk order (an exclusive
// scan of their chunk counts), each warp takes a contiguous range of chunks
// and each lane one chunk of it, so that every lane has work and a warp
// reads consecutive chunks of the same rows.  A lane finds its row from the
// row starts that fall inside its warp's 32-chunk window (a ballot over the
// next 32 rows, which is enough because every listed row is nonempty; empty
// rows are settled while listing).  The lanes of one row combine their
// fixed-point sums by a segmented shuffle reduction, and the first lane of
// each row segment adds it to the row's shared accumulator.  The sums are
// integers, so the result does not depend on how the rows are split: it is
// the row walk's, bit for bit.
template <int NT>
__device__ void count_rows_group_chunks(const RowArgs<ModeF32>& A, int b, unsigned char* smem, int* s_n)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr unsigned long long ONE = 2147483648ull;  // one neighbour inside r_l, in units of 2^-31
    const CountLayout ly = count_layout(A.cp, sizeof(int4));
    int4* spos = (int4*)smem;
    int* plist = (int*)(smem + ly.plist);
    int* cstart = (int*)(smem + ly.cstart);
    unsigned long long* acc = (unsigned long long*)(smem + ly.acc);
    __shared__ int s_wsum[NT / 32];
    int* bad = &A.st->bad_index;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    __syncthreads();  // the previous group is done with the shared arrays
    const int p0 = __ldg(A.G.cell_start + OWN_CELLS * b);
    const int n_own = __ldg(A.G.cell_start + OWN_CELLS * b + OWN_CELLS) - p0;
    // the unsettled own particles (s'_i = NaN from k_count_near); an empty row is settled here
    const int nl = list_own<NT>(n_own, plist, s_n, A.cp.omax, bad, [&](int j) {
        if (!isnan(A.ds[p0 + j])) return false;
        if (row_len(__ldg(A.nnb + p0 + j)) > 0) return true;
        finish_count_fix(A, p0 + j, 0ull);
        return false;
    });
    if (nl == 0) return;
    // the count reads no s_j, so the spare word of a staged position holds its residuals
    stage_by_table<NT>(A.aux.stage_idx + (size_t)b * A.cp.smax, __ldg(A.aux.meta + b).x, A.cp.smax, A.n, bad,
                       [&](int m, int jj) {
                           int4 pj = A.pos[jj];
                           pj.w = resid_of(A, jj);
                           spos[m] = pj;
                       });
    // chunk counts -> first chunk of each row: each thread scans a contiguous run of rows
    const int per = (nl + NT - 1) / NT;
    const int u0 = min(nl, t * per), u1 = min(nl, u0 + per);
    int loc = 0;
    for (int u = u0; u < u1; ++u) {
        const int nch = (row_len(__ldg(A.nnb + p0 + plist[u])) + 3) >> 2;
        cstart[u] = nch;
        loc += nch;
    }
    int inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    int run = inc - loc, total = 0;
    for (int w = 0; w < NT / 32; ++w) {
        const int v = s_wsum[w];
        if (w < warp) run += v;
        total += v;
    }
    for (int u = u0; u < u1; ++u) {
        const int nch = cstart[u];
        cstart[u] = run;
        run += nch;
        acc[u] = 0ull;
    }
    if (t == 0) cstart[nl] = total;
    __syncthreads();
    // this warp's chunks [c_begin, c_end); r_prev is the row holding chunk c0 - 1 (-1 before the first)
    const int cw = (total + NT / 32 - 1) / (NT / 32);
    const int c_begin = min(total, warp * cw), c_end = min(total, c_begin + cw);
    int r_prev;
    {
        int lo = 0, hi = nl;  // rows whose first chunk is below c_begin
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cstart[mid] < c_begin) lo = mid + 1;
            else hi = mid;
        }
        r_prev = lo - 1;
    }
    const Coef& c = A.c;
    for (int c0 = c_begin; c0 < c_end; c0 += 32) {
        // rows starting inside [c0, c0 + 32): r_prev + 1 .. r_prev + k (rows are nonempty)
        const int cand = r_prev + 1 + lane;
        const int cs = cand < nl ? cstart[cand] : INT_MAX;
        const bool starts = (unsigned)(cs - c0) < 32u;
        const unsigned bits = __reduce_or_sync(FULL, starts ? 1u << (cs - c0) : 0u);
        int u = r_prev + __popc(bits & (FULL >> (31 - lane)));  // row of chunk c0 + lane
        r_prev += __popc(__ballot_sync(FULL, starts));
        const int ch = c0 + lane;
        unsigned long long a = 0ull;
        if (ch >= c_end) {
            u = -1;
        } else if ((unsigned)u >= (unsigned)nl) {
            *bad = BAD_STAGING_SIZE;
            u = -1;
        } else {
            const int p = p0 + plist[u];
            const int4 pi = A.pos[p];
            const int ri = resid_of(A, p);
            const int len = row_len(__ldg(A.nnb + p));
            const int e0 = 4 * (ch - cstart[u]);
            int h[4];
            unpack4(__ldg(reinterpret_cast<const uint2*>(A.nbr + (size_t)p * A.cp.cap + e0)), h);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (e0 + k >= len) break;
                const int4 pj = spos[checked_staged(h[k], A.cp.smax, bad)];
                const unsigned long long r2 = r2_fix(pi, pj);
                if (r2 < c.rh2_fix) {
                    if (r2 <= c.rl2_fix) {
                        a += ONE;
                    } else {
                        // omega has zero slope at both ends of the window, so a pair that the
                        // finer separation moves across r_l or r_h changes n_i by O(dr^2)
                        const unsigned long long rf = r2_fine(pi, ri, pj, pj.w, r2);
                        if (rf <= c.rl2_fix) a += ONE;
                        else if (rf < c.rh2_fix) a += window_weight_tab(rf - c.rl2_fix, c.wtab, c.wsh);
                    }
                }
            }
        }
        // segmented sum over the lanes of each row (a row's lanes are contiguous): after the
        // step of width o a lane holds the sum over [lane, lane + 2o) within its row
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_down_sync(FULL, a, o);
            const int uy = __shfl_down_sync(FULL, u, o);
            if (lane + o < 32 && uy == u) a += y;
        }
        const int up = __shfl_up_sync(FULL, u, 1);
        if (u >= 0 && (lane == 0 || up != u)) atomicAdd(&acc[u], a);
    }
    __syncthreads();
    for (int u = t; u < nl; u += NT) finish_count_fix(A, p0 + plist[u], acc[u]);
}

// Dense mode of the count walk: more than n / DENSE_DIV unsettled particles.
template <class M>
__device__ __forceinline__ bool count_rows_dense(const RowArgs<M>& A) { return A.st->nu > A.n / DENSE_DIV; }

template <class M, int NT>
__global__ void __launch_bounds__(NT) k_count_rows(RowArgs<M> A, int ngroups, int tmax)
{
    // the list this step's counts used is current: clear the request (after both close counts)
    if (blockIdx.x == 0 && threadIdx.x == 0) A.st->rebuild = 0;
    if (halted(A.st)) return;
    if (!count_rows_dense(A)) {
        const int nu = A.st->nu;
        for (int k = blockIdx.x * (NT / 32) + (threadIdx.x >> 5); k < nu; k += gridDim.x * (NT / 32))
            count_rows_item(A, k);
        return;
    }
    __shared__ int s_n;
    extern __shared__ __align__(16) unsigned char smem[];
    for (int b = blockIdx.x; b < ngroups; b += gridDim.x) count_rows_group<M, NT>(A, b, tmax, smem, &s_n);
}

// ================================================================ chain-rule pass
// A_i = s'_i sum_j s_j V_a(r_ij) for the particles inside the switching
// window (s'_i != 0), which k_count_rows listed.  In the sparse mode every
// list neighbour of a window particle loses its whole-force tag (its window
// term needs A_i) and joins the general list of k_force_rows.  In the dense
// mode nearly every particle neighbours a window particle, so no tag is
// cleared: k_force_rows, which makes the same mode test, then takes every
// particle.
template <class M, class Walk, class Fetch>
__device__ __forceinline__ typename M::real chain_row(const typename M::pos_t& pi, Walk&& walk, int width,
                                                      Fetch&& fetch, const Coef& c, const Geom& g)
{
    using real = typename M::real;
    real acc = 0;
    walk([&](int m) {
        const auto pj = fetch(m);
        if constexpr (M::fp64) {
            const double r2 = r2_d<M>(pi, pj, g);
            if (r2 > c.rr2 && r2 < c.ra2) acc = __fma_rn(get_s(pj), Va_d(sqrt(r2), c), acc);
        } else {
            const unsigned long long r2i = r2_fix(pi, pj);
            if (r2i > c.rr2_fix && r2i < c.ra2_fix) {
                // spelt-out products and sums (no contraction that could differ between kernels)
                const float r2 = __fmul_rn(u64_to_float(r2i), g.s32sq);
                const float r = __fmul_rn(r2, rsqrtf(r2));
                const float uu = __fdividef(__fmul_rn(s64_to_float((long long)r2i - (long long)c.rm2_fix), c.s2hinv),
                                            __fadd_rn(r, c.rmf));
                const float q = __fmaf_rn(-uu, uu, 1.0f);
                acc = __fmaf_rn(get_s(pj), __fmul_rn(__fmul_rn(-c.Eaf, q), q), acc);
            }
        }
    });
    return group_sum(acc, width);
}

// Sparse chain-rule term: window particle k of the list k_count_rows made (one
// warp, one lane per row entry); clears the whole-force tag of every list
// neighbour, which then joins the general list of k_force_rows.
template <class M>
__device__ __forceinline__ void chain_item(const RowArgs<M>& A, int k)
{
    using real = typename M::real;
    const int p = A.wpart[k];
    const LaneRow lr = lane_row(A.nbr, p, A.cp.cap);
    const int b = __ldg(A.aux.grp + p);
    const int* sidx = A.aux.stage_idx + (size_t)b * A.cp.smax;
    const int len = row_len(__ldg(A.nnb + p));
    const real acc = chain_row<M>(A.pos[p], [&](auto&& v) { walk_lanes_from(lr, len, v); }, 32, [&](int m) {
        const int jj = table_index(A, sidx, m);
        // the force of jj needs A_i: if it was tagged whole, it now goes on the general list
        if constexpr (!M::fp64) {
            if (atomicExch(reinterpret_cast<float*>(static_cast<float4*>(A.aux.fcore) + jj) + 3, 0.0f) != 0.0f)
                list_append(A.aux.glist, &A.st->ngen, jj);
        }
        return A.pos[jj];
    }, A.c, A.g);
    if ((threadIdx.x & 31) == 0) A.sA[p].y = A.ds[p] * acc;
}

// Dense chain-rule terms of cell group b: its own window particles (whole
// block; starts with a block barrier).
template <class M, int NT>
__device__ __forceinline__ void chain_group(const RowArgs<M>& A, int b, int tmax, unsigned char* smem, int* s_n)
{
    using pos_t = typename M::pos_t;
    using real = typename M::real;
    const DenseLayout ly = dense_layout(A.cp, sizeof(pos_t), 0);
    pos_t* spos = (pos_t*)smem;
    int* plist = (int*)(smem + ly.plist);
    __syncthreads();  // the previous group is done with the shared arrays
    const int p0 = __ldg(A.G.cell_start + OWN_CELLS * b);
    const int n_own = __ldg(A.G.cell_start + OWN_CELLS * b + OWN_CELLS) - p0;
    const int nl = list_own<NT>(n_own, plist, s_n, A.cp.omax, &A.st->bad_index,
                                [&](int j) { return A.ds[p0 + j] != (real)0; });
    if (nl == 0) return;
    stage_by_table<NT>(A.aux.stage_idx + (size_t)b * A.cp.smax, __ldg(A.aux.meta + b).x, A.cp.smax, A.n,
                       &A.st->bad_index, [&](int m, int jj) { spos[m] = A.pos[jj]; });
    __syncthreads();
    dense_rounds<NT>(nl, tmax, [&](int u, int sub, int tpp) {
        const bool act = u < nl;
        const int p = p0 + (act ? plist[u] : 0);
        const uint16_t* row = A.nbr + (size_t)p * A.cp.cap;
        const int len = act ? row_len(__ldg(A.nnb + p)) : 0;
        const real acc = chain_row<M>(A.pos[p], [&](auto&& v) { walk_chunks(row, len, sub, tpp, v); }, tpp,
                                      [&](int m) { return spos[checked_staged(m, A.cp.smax, &A.st->bad_index)]; },
                                      A.c, A.g);
        if (act && sub == 0) A.sA[p].y = A.ds[p] * acc;
    });
}

template <class M>
__device__ __forceinline__ bool chain_dense(const RowArgs<M>& A) { return A.st->nwin > A.n / DENSE_DIV; }

template <class M, int NT>
__global__ void __launch_bounds__(NT) k_chain(RowArgs<M> A, int ngroups, int tmax)
{
    wait_for_predecessor();
    if (halted(A.st)) return;
    if (!chain_dense(A)) {
        const int nw = A.st->nwin;
        for (int k = blockIdx.x * (NT / 32) + (threadIdx.x >> 5); k < nw; k += gridDim.x * (NT / 32)) chain_item(A, k);
        return;
    }
    __shared__ int s_n;
    extern __shared__ __align__(16) unsigned char smem[];
    for (int b = blockIdx.x; b < ngroups; b += gridDim.x) chain_group<M, NT>(A, b, tmax, smem, &s_n);
}

// ================================================================ pass 2: forces + BAOAB
// k_force_rows: the whole force of every particle without a tagged whole
// force (not saturated, a neighbour of a window particle, more near entries
// than the close list holds, or any particle in the FP64 mode), every term
// of its full row; neighbours carry s_j in the positions' spare word.  When
// k_chain ran dense (it cleared no tags) every particle is taken.  The
// result overwrites the particle's force slot with the tag set.
template <class M, class Walk, class Fetch>
__device__ __forceinline__ void force_row(const typename M::pos_t& pi, typename M::real si, typename M::real Ai,
                                          Walk&& walk, int width, Fetch&& fetch, const Coef& c, const Geom& g,
                                          typename M::real f[3])
{
    using real = typename M::real;
    real fx = 0, fy = 0, fz = 0;
    walk([&](int m) {
        real Aj;
        const auto pj = fetch(m, Aj);
        if constexpr (M::fp64) pair_f64(pi, si, Ai, pj, get_s(pj), Aj, c, g, fx, fy, fz);
        else pair_f32(pi, si, Ai, pj, get_s(pj), Aj, c, g, fx, fy, fz);
    });
    f[0] = group_sum(fx, width);
    f[1] = group_sum(fy, width);
    f[2] = group_sum(fz, width);
}

template <class M>
__device__ __forceinline__ void force_out(void* fcore, int p, const typename M::real f[3])
{
    if constexpr (M::fp64) static_cast<F64x4*>(fcore)[p] = F64x4{f[0], f[1], f[2], 1.0};
    else static_cast<float4*>(fcore)[p] = make_float4(f[0], f[1], f[2], 1.0f);
}

template <class M>
__device__ __forceinline__ bool tagged_whole(const void* fcore, int p)
{
    if constexpr (M::fp64) return static_cast<const F64x4*>(fcore)[p].w != 0.0;
    else return static_cast<const float4*>(fcore)[p].w != 0.0f;
}

// The force walk runs dense when k_chain did (it then cleared no tag, and
// every particle is taken) or when the general list is long.
template <class M>
__device__ __forceinline__ bool force_all(const RowArgs<M>& A) { return A.st->nwin > A.n / DENSE_DIV; }
template <class M>
__device__ __forceinline__ bool force_dense(const RowArgs<M>& A)
{
    return force_all(A) || A.st->ngen > A.n / DENSE_DIV;
}

// Sparse force: general particle k (one warp, one lane per row entry).
template <class M>
__device__ __forceinline__ void force_item(const RowArgs<M>& A, int k)
{
    using pos_t = typename M::pos_t;
    using real = typename M::real;
    const bool useA = A.st->nwin > 0;  // A_j != 0 only for window particles
    const int p = A.aux.glist[k];
    const LaneRow lr = lane_row(A.nbr, p, A.cp.cap);
    const int b = __ldg(A.aux.grp + p);
    const int* sidx = A.aux.stage_idx + (size_t)b * A.cp.smax;
    const int len = row_len(__ldg(A.nnb + p));
    const pos_t pi = A.pos[p];
    real f[3];
    force_row<M>(pi, get_s(pi), useA ? A.sA[p].y : (real)0, [&](auto&& v) { walk_lanes_from(lr, len, v); }, 32,
                 [&](int m, real& Aj) {
                     const int jj = table_index(A, sidx, m);
                     Aj = useA ? A.sA[jj].y : (real)0;
                     return A.pos[jj];
                 },
                 A.c, A.g, f);
    if ((threadIdx.x & 31) == 0) force_out<M>(A.aux.fcore, p, f);
}

// Dense forces of cell group b: its own particles without a whole-force tag,
// all of them after a dense chain-rule pass (whole block; starts with a block
// barrier).
template <class M, int NT>
__device__ __forceinline__ void force_group(const RowArgs<M>& A, int b, int tmax, unsigned char* smem, int* s_n)
{
    using pos_t = typename M::pos_t;
    using real = typename M::real;
    const bool useA = A.st->nwin > 0;
    const bool all = force_all(A);
    const DenseLayout ly = dense_layout(A.cp, sizeof(pos_t), sizeof(real));
    pos_t* spos = (pos_t*)smem;
    real* sAj = (real*)(smem + ly.extra);
    int* plist = (int*)(smem + ly.plist);
    __syncthreads();  // the previous group is done with the shared arrays
    const int p0 = __ldg(A.G.cell_start + OWN_CELLS * b);
    const int n_own = __ldg(A.G.cell_start + OWN_CELLS * b + OWN_CELLS) - p0;
    int nl;
    if (all) {
        nl = min(n_own, A.cp.omax);
        if (n_own > A.cp.omax && threadIdx.x == 0) A.st->bad_index = BAD_STAGING_SIZE;
        for (int j = threadIdx.x; j < nl; j += NT) plist[j] = j;
    } else {
        nl = list_own<NT>(n_own, plist, s_n, A.cp.omax, &A.st->bad_index,
                          [&](int j) { return !tagged_whole<M>(A.aux.fcore, p0 + j); });
    }
    if (nl == 0) return;
    stage_by_table<NT>(A.aux.stage_idx + (size_t)b * A.cp.smax, __ldg(A.aux.meta + b).x, A.cp.smax, A.n,
                       &A.st->bad_index, [&](int m, int jj) {
                           spos[m] = A.pos[jj];
                           sAj[m] = useA ? A.sA[jj].y : (real)0;
                       });
    __syncthreads();
    dense_rounds<NT>(nl, tmax, [&](int u, int sub, int tpp) {
        const bool act = u < nl;
        const int p = p0 + (act ? plist[u] : 0);
        const uint16_t* row = A.nbr + (size_t)p * A.cp.cap;
        const int len = act ? row_len(__ldg(A.nnb + p)) : 0;
        const pos_t pi = A.pos[p];
        real f[3];
        force_row<M>(pi, get_s(pi), useA ? A.sA[p].y : (real)0,
                     [&](auto&& v) { walk_chunks_padded(row, len, sub, tpp, v); }, tpp,
                     [&](int m, real& Aj) {
                         m = checked_staged(m, A.cp.smax, &A.st->bad_index);
                         Aj = sAj[m];
                         return spos[m];
                     },
                     A.c, A.g, f);
        if (act && sub == 0) force_out<M>(A.aux.fcore, p, f);
    });
}

template <class M, int NT>
__global__ void __launch_bounds__(NT) k_force_rows(RowArgs<M> A, int ngroups, int tmax)
{
    wait_for_predecessor();
    if (halted(A.st)) return;
    if (!force_dense(A)) {
        const int ng = A.st->ngen;
        for (int k = blockIdx.x * (NT / 32) + (threadIdx.x >> 5); k < ng; k += gridDim.x * (NT / 32)) force_item(A, k);
        return;
    }
    __shared__ int s_n;
    extern __shared__ __align__(16) unsigned char smem[];
    for (int b = blockIdx.x; b < ngroups; b += gridDim.x) force_group<M, NT>(A, b, tmax, smem, &s_n);
}

// k_step: the BAOAB update of every particle from its force slot (or, for a
// force evaluation, the forces in caller order).  A streaming kernel.
template <class M, int EPI>
__device__ __forceinline__ void step_item(int p, int n, const Geom& g, const GroupAux& aux, const int* __restrict__ id,
                                          typename M::pos_t* __restrict__ pos_next,
                                          const typename M::pos_t* __restrict__ xref, const StepArgs& a, Status* st)
{
    typename M::real f[3];
    if constexpr (M::fp64) {
        const F64x4 fc = static_cast<const F64x4*>(aux.fcore)[p];
        f[0] = fc.x;
        f[1] = fc.y;
        f[2] = fc.z;
    } else {
        const float4 fc = static_cast<const float4*>(aux.fcore)[p];
        f[0] = fc.x;
        f[1] = fc.y;
        f[2] = fc.z;
    }
    PState<M> q;
    load_pstate<M, EPI>(p, n, a, id, xref, q);
    if constexpr (EPI == EPI_FORCE) {
        if (a.F_out) {
            const size_t o = 3 * (size_t)q.id;
            a.F_out[o + 0] = (double)f[0];
            a.F_out[o + 1] = (double)f[1];
            a.F_out[o + 2] = (double)f[2];
        }
    } else {
        integrate<M, EPI>(p, n, g, f[0], f[1], f[2], a, q, st, pos_next);
    }
}

template <class M, int EPI>
__global__ void __launch_bounds__(TPB) k_step(int n, Geom g, GroupAux aux, const int* __restrict__ id,
                                              typename M::pos_t* __restrict__ pos_next,
                                              const typename M::pos_t* __restrict__ xref, StepArgs a, Status* st)
{
    wait_for_predecessor();
    if (halted(st)) return;
    // An update that opens a step empties the work lists of the next iteration (their readers,
    // the row walks, are done); the last update of a call keeps them for the statistics.
    if constexpr (EPI == EPI_START || EPI == EPI_FINISH_START) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->nwin = 0;
            st->nu = 0;
            st->ngen = 0;
        }
    }
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) step_item<M, EPI>(p, n, g, aux, id, pos_next, xref, a, st);
}

// ================================================================ FP64 energy / virial
// Requested energies are held to 1e-9 relative, which needs the switching
// factors to FP64 accuracy: the counts, s, s' and A are recomputed here in
// FP64 from the exact fixed-point separations (these kernels run only when U
// or W is asked for, never inside the step loop).  One block per cell group,
// one thread per own particle.
template <class M>
__global__ void __launch_bounds__(SC_TPB) k_count_e(Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                    SuperGrid G, SuperCaps cp, const uint16_t* __restrict__ nbr,
                                                    const int* __restrict__ nnb, double2* __restrict__ sd,
                                                    double* __restrict__ n_sorted, const Status* st)
{
    using pos_t = typename M::pos_t;
    if (halted(st)) return;
    __shared__ SuperTab T;
    extern __shared__ __align__(16) unsigned char smem[];
    int p0, n_own, total;
    load_group(blockIdx.x, g, G, T, p0, n_own, total);
    pos_t* spos = (pos_t*)smem;
    stage<pos_t>(T, total, [&](int j) { return pos[j]; }, [&](int m, const pos_t& v) { spos[m] = v; });
    __syncthreads();
    for (int j = threadIdx.x; j < n_own; j += SC_TPB) {
        const int p = p0 + j;
        const int len = row_len(nnb[p]);
        const pos_t pi = pos[p];
        double acc = 0.0;
        for (int e = 0; e < len; ++e) {
            const double r2 = r2_d<M>(pi, spos[nbr[(size_t)p * cp.cap + e]], g);
            if (r2 < c.rh2) acc += r2 <= c.rl2 ? 1.0 : omega_d(sqrt(r2), c.r_l, c.r_h);
        }
        sd[p] = make_double2(omega_d(acc, c.fd, c.fd + 1.0), domega_d(acc, c.fd, c.fd + 1.0));
        if (n_sorted) n_sorted[p] = acc;
    }
}

template <class M>
__global__ void __launch_bounds__(SC_TPB) k_chain_e(Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                    SuperGrid G, SuperCaps cp, const uint16_t* __restrict__ nbr,
                                                    const int* __restrict__ nnb, const double2* __restrict__ sd,
                                                    double* __restrict__ Ad, const Status* st)
{
    using pos_t = typename M::pos_t;
    if (halted(st)) return;
    __shared__ SuperTab T;
    extern __shared__ __align__(16) unsigned char smem[];
    int p0, n_own, total;
    load_group(blockIdx.x, g, G, T, p0, n_own, total);
    const PassLayout ly = pass_layout(cp, sizeof(pos_t), sizeof(double));
    pos_t* spos = (pos_t*)smem;
    double* ss = (double*)(smem + ly.val);
    struct PS {
        pos_t p;
        double s;
    };
    stage<PS>(
        T, total, [&](int j) { return PS{pos[j], sd[j].x}; },
        [&](int m, const PS& v) {
            spos[m] = v.p;
            ss[m] = v.s;
        });
    __syncthreads();
    for (int j = threadIdx.x; j < n_own; j += SC_TPB) {
        const int p = p0 + j;
        const double dsi = sd[p].y;
        if (dsi == 0.0) {
            Ad[p] = 0.0;
            continue;
        }
        const int len = row_len(nnb[p]);
        const pos_t pi = pos[p];
        double acc = 0.0;
        for (int e = 0; e < len; ++e) {
            const int m = nbr[(size_t)p * cp.cap + e];
            const double r2 = r2_d<M>(pi, spos[m], g);
            if (r2 > c.rr2 && r2 < c.ra2) acc += ss[m] * Va_d(sqrt(r2), c);
        }
        Ad[p] = dsi * acc;
    }
}

// Per-block partial sums of U = sum_{i<j} [V_r + s_i s_j V_a], W = sum_{i<j} -g r
// and of the number of pairs with r < r_c, each pair seen from both ends (halves).
template <class M>
__global__ void __launch_bounds__(SC_TPB) k_energy(Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                   SuperGrid G, SuperCaps cp, const uint16_t* __restrict__ nbr,
                                                   const int* __restrict__ nnb, const double2* __restrict__ sd,
                                                   const double* __restrict__ Ad, double* __restrict__ partial,
                                                   long long* __restrict__ ppairs, const Status* st)
{
    using pos_t = typename M::pos_t;
    __shared__ SuperTab T;
    __shared__ double se[SC_TPB], sw[SC_TPB];
    __shared__ long long sp[SC_TPB];
    extern __shared__ __align__(16) unsigned char smem[];
    const PassLayout ly = pass_layout(cp, sizeof(pos_t), sizeof(double2));
    pos_t* spos = (pos_t*)smem;
    double2* ssa = (double2*)(smem + ly.val);  // (s_j, A_j)
    double e = 0.0, w = 0.0;
    long long pairs = 0;
    if (!halted(st)) {
        int p0, n_own, total;
        load_group(blockIdx.x, g, G, T, p0, n_own, total);
        struct PS {
            pos_t p;
            double2 sa;
        };
        stage<PS>(
            T, total, [&](int j) { return PS{pos[j], make_double2(sd[j].x, Ad[j])}; },
            [&](int m, const PS& v) {
                spos[m] = v.p;
                ssa[m] = v.sa;
            });
        __syncthreads();
        for (int j = threadIdx.x; j < n_own; j += SC_TPB) {
            const int p = p0 + j;
            const int len = row_len(nnb[p]);
            const pos_t pi = pos[p];
            const double si = sd[p].x, Ai = Ad[p];
            for (int k = 0; k < len; ++k) {
                const int m = nbr[(size_t)p * cp.cap + k];
                const double r2 = r2_d<M>(pi, spos[m], g);
                if (r2 >= c.rc2) continue;
                ++pairs;
                const double sjv = ssa[m].x, Aj = ssa[m].y;
                const double r = sqrt(r2);
                e += 0.5 * (Vr_d(r2, c) + si * sjv * Va_d(r, c));
                const double gg = dVr_over_r_d(r2, c) * r + si * sjv * dVa_d(r, c) + (Ai + Aj) * domega_d(r, c.r_l, c.r_h);
                w += 0.5 * (-gg * r);
            }
        }
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    sp[threadIdx.x] = pairs;
    __syncthreads();
    for (int s = SC_TPB / 2; s > 0; s >>= 1) {
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


// ================================================================ valency observables
// z_i = #{j != i : r_ij < r_a} (Sec. 3: neighbours within the attraction
// range, an instantaneous and strict distance criterion), walked over the
// particle's list row (radius r_c + skin >= r_a).  Integer sums only: acc[0]
// = sum of z, acc[1] = particles with z > f, acc[2 + k] = particles with
// z = k (last bin: z >= ZHIST - 1), each formed per block in shared memory
// and added once per block.  Optional z per particle in caller order.
constexpr int ZHIST = 32;
template <class M>
__global__ void __launch_bounds__(TPB) k_observe(int n, Geom g, Coef c, const typename M::pos_t* __restrict__ pos,
                                                 SuperCaps cp, GroupAux aux, const uint16_t* __restrict__ nbr,
                                                 const int* __restrict__ nnb, const int* __restrict__ id,
                                                 int* __restrict__ z_out, unsigned long long* __restrict__ acc,
                                                 const Status* st)
{
    __shared__ unsigned long long s_acc[2 + ZHIST];
    for (int k = threadIdx.x; k < 2 + ZHIST; k += blockDim.x) s_acc[k] = 0ull;
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && !halted(st)) {
        const int b = __ldg(aux.grp + p);
        const int* sidx = aux.stage_idx + (size_t)b * cp.smax;
        const int len = row_len(__ldg(nnb + p));
        const uint16_t* row = nbr + (size_t)p * cp.cap;
        const typename M::pos_t pi = pos[p];
        int z = 0;
        for (int e = 0; e < len; ++e) {
            const typename M::pos_t pj = pos[__ldg(sidx + __ldg(row + e))];
            if constexpr (M::fp64) z += r2_d<M>(pi, pj, g) < c.ra2;
            else z += r2_fix(pi, pj) < c.ra2_fix;
        }
        if (z_out) z_out[id[p]] = z;
        atomicAdd(&s_acc[0], (unsigned long long)z);
        if ((double)z > c.f) atomicAdd(&s_acc[1], 1ull);
        atomicAdd(&s_acc[2 + min(z, ZHIST - 1)], 1ull);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 + ZHIST; k += blockDim.x)
        if (s_acc[k]) atomicAdd(acc + k, s_acc[k]);
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

// Per-particle sums of the thermodynamic reductions (vbc_compute_thermo):
// KE = sum_i |v_i|^2 / 2 from the state (unit mass), sum_i n_i from FP64
// counts nv[0..n), and the particles inside their switching window
// (dsv[i * ds_stride] != 0).  A fixed grid takes the particles in a
// grid-stride loop and each block writes its partial sums, so the result
// depends on n and the state alone.
constexpr int THERMO_GRID = 592;  // 4 blocks of RED_TPB per SM of a B300
struct ThermoOut {
    double ke, nsum;
    long long win;
};
template <class M>
__global__ void __launch_bounds__(RED_TPB) k_thermo_part(int n, const void* __restrict__ v,
                                                         const double* __restrict__ nv,
                                                         const double* __restrict__ dsv, int ds_stride,
                                                         double* __restrict__ part, long long* __restrict__ wpart)
{
    __shared__ double sk[RED_TPB], sn[RED_TPB];
    __shared__ long long sw[RED_TPB];
    double ke = 0.0, ns = 0.0;
    long long w = 0;
    for (int p = blockIdx.x * RED_TPB + threadIdx.x; p < n; p += gridDim.x * RED_TPB) {
        double v2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double vd;
            if constexpr (M::fp64) vd = ((const double*)v)[(size_t)d * n + p];
            else vd = (double)((const long long*)v)[(size_t)d * n + p] * 9.094947017729282e-13;  // 2^-40
            v2 += vd * vd;
        }
        ke += 0.5 * v2;
        ns += nv[p];
        w += dsv[(size_t)p * ds_stride] != 0.0 ? 1 : 0;
    }
    sk[threadIdx.x] = ke;
    sn[threadIdx.x] = ns;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int s = RED_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sk[threadIdx.x] += sk[threadIdx.x + s];
            sn[threadIdx.x] += sn[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sk[0];
        part[2 * blockIdx.x + 1] = sn[0];
        wpart[blockIdx.x] = sw[0];
    }
}

// Fixed-order sum of the THERMO_GRID block partials.
__global__ void __launch_bounds__(RED_TPB) k_thermo_final(int nb, const double* __restrict__ part,
                                                          const long long* __restrict__ wpart, ThermoOut* out)
{
    __shared__ double sk[RED_TPB], sn[RED_TPB];
    __shared__ long long sw[RED_TPB];
    double ke = 0.0, ns = 0.0;
    long long w = 0;
    for (int b = threadIdx.x; b < nb; b += RED_TPB) {
        ke += part[2 * b];
        ns += part[2 * b + 1];
        w += wpart[b];
    }
    sk[threadIdx.x] = ke;
    sn[threadIdx.x] = ns;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int s = RED_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sk[threadIdx.x] += sk[threadIdx.x + s];
            sn[threadIdx.x] += sn[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = ThermoOut{sk[0], sn[0], sw[0]};
}

// ================================================================ state I/O
// Caller order [n][3] doubles -> internal state in sorted order, and the
// fixed-point words.  FP32 mode: X = round(x 2^52 / L) and V = round(v 2^40)
// (int64), which hold |x| < 1024 L and |v| < 2^22; a value beyond that, or a
// non-finite one (which the integer state could not carry), raises bad_input
// and halts the system until the next load.
template <class M>
__global__ void __launch_bounds__(TPB) k_load_state(int n, Geom g, const double* __restrict__ pos_in,
                                                    const double* __restrict__ vel_in, const int* __restrict__ id,
                                                    void* __restrict__ xs, void* __restrict__ vs,
                                                    typename M::pos_t* __restrict__ pos, int* __restrict__ resid,
                                                    const typename M::pos_t* __restrict__ xref, float half_skin2,
                                                    Status* st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = id[i];
    bool bad = false;
    float d2 = 0.0f;  // squared distance from the position at the last list build
    if constexpr (M::fp64) {
        double xx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xx[d] = pos_in[3 * (size_t)o + d];
            const double v = vel_in ? vel_in[3 * (size_t)o + d] : 0.0;
            bad |= !isfinite(xx[d]) || !isfinite(v);
            ((double*)xs)[(size_t)d * n + i] = xx[d];
            ((double*)vs)[(size_t)d * n + i] = v;
        }
        const P64 pn = ModeF64::from_x(xx[0], xx[1], xx[2], g);
        pos[i] = pn;
        const P64 pr = xref[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float u = (float)(int)(ModeF64::hi32(pn, d) - ModeF64::hi32(pr, d)) * (float)g.s32d[d];
            d2 += u * u;
        }
    } else {
        int w[3];
        long long Ps[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double xf = pos_in[3 * (size_t)o + d] * g.inv32[d] * 1048576.0;  // x 2^52 / L
            const double vf = (vel_in ? vel_in[3 * (size_t)o + d] : 0.0) * 1099511627776.0;  // v 2^40
            bad |= !(fabs(xf) < 4611686018427387904.0) || !(fabs(vf) < 4611686018427387904.0);  // 2^62
            const long long P = bad ? 0ll : __double2ll_rn(xf);
            ((long long*)xs)[(size_t)d * n + i] = P;
            Ps[d] = P;
            w[d] = ModeF32::word(P);
            ((long long*)vs)[(size_t)d * n + i] = bad ? 0ll : __double2ll_rn(vf);
        }
        pos[i] = make_int4(w[0], w[1], w[2], 0);
        resid[i] = pack_resid3(Ps[0], Ps[1], Ps[2]);
        const int4 pr = xref[i];
        const float ux = (float)(w[0] - pr.x) * g.s32, uy = (float)(w[1] - pr.y) * g.s32,
                    uz = (float)(w[2] - pr.z) * g.s32;
        d2 = ux * ux + uy * uy + uz * uz;
    }
    if (bad) st->bad_input = 1;
    // the list stays valid while every particle is within skin / 2 of its position at the build
    if (bad || !(d2 <= half_skin2)) st->rebuild = 1;
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
            v = (double)((const long long*)vs)[(size_t)d * n + i] * 9.094947017729282e-13;  // 2^-40
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


// Lists in caller indices (diagnostics): staging index -> sorted index -> id.
__global__ void __launch_bounds__(SC_TPB) k_store_nlist(Geom g, SuperGrid G, SuperCaps cp,
                                                        const uint16_t* __restrict__ nbr, const int* __restrict__ nnb,
                                                        const int* __restrict__ id, int cap_out,
                                                        int* __restrict__ nnb_out, int* __restrict__ nbr_out)
{
    __shared__ SuperTab T;
    int p0, n_own, total;
    load_group(blockIdx.x, g, G, T, p0, n_own, total);
    for (int j = threadIdx.x; j < n_own; j += SC_TPB) {
        const int p = p0 + j;
        const int o = id[p];
        const int len = row_len(nnb[p]);
        if (nnb_out) nnb_out[o] = len;
        if (!nbr_out) continue;
        for (int e = 0; e < len && e < cap_out; ++e)
            nbr_out[(size_t)o * cap_out + e] = id[staged_index(T, nbr[(size_t)p * cp.cap + e])];
    }
}


// Opens one loop iteration: advances the device iteration counter (which
// keys the Langevin noise) and, inside a CUDA graph, sets the conditional
// that runs the rebuild body only when a rebuild is due; clears the list of
// window particles that the iteration's count fills.
// The gate of a loop iteration: advances the iteration counter and, in a graph,
// opens the rebuild conditional.  reset clears the work-list counters here; a
// graph whose close count runs beside the conditional (not after this gate)
// has them cleared by the previous update (k_step) or by k_set_iter instead.
__global__ void k_gate(Status* st, cudaGraphConditionalHandle h, int in_graph, int reset)
{
    st->iter += 1;
    if (reset) {
        st->nwin = 0;
        st->nu = 0;
        st->ngen = 0;
    }
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
    st->nwin = 0;  // the work lists of the first iteration start empty
    st->nu = 0;
    st->ngen = 0;
}

__global__ void k_iota(int n, int* __restrict__ id)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = i;
}

}  // namespace vbc
