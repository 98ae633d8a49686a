// vbc_batch.cuh -- one persistent launch per loop iteration for many systems.
//
// A batch of independent systems (parameter sweeps, Sec. 5) advances with one
// cooperative launch per Langevin iteration.  The launch runs the iteration's
// phases in order -- gate, the list rebuild of every system that needs one,
// the close count, the count, chain-rule and force row walks, the update --
// and each phase takes the work items of all systems together: particles,
// cells, scan chunks, cell groups or list entries, numbered system after
// system.  A grid-wide wait separates the phases.  Every item runs the same
// device function as the single-system kernels (vbc_kernels.cuh), so each
// system's result is bitwise the one it gets stepped alone.
//
// The grid-wide waits are bounded: a block that has waited wait_limit spins
// for the others gives up, raises the batch's timeout flag and returns, and
// every block that sees the flag after a wait returns too.  Work already done
// stays consistent (a phase starts only once every block finished the one
// before), but the iteration is incomplete: the host reports VBC_ERR_TIMEOUT
// and halts the batch's systems until their state is set again.
#pragma once

#include "vbc_kernels.cuh"

namespace vbc {

// Control words of one batch: the grid-wide wait and its outcome.
struct BatchCtl {
    unsigned int count;    // blocks arrived at the current wait
    unsigned int gen;      // completed waits
    int timeout;           // 1: a wait gave up
    int any_due;           // 1: some system rebuilds its list in this iteration
    long long wait_limit;  // spins (of about 100 ns) before a wait gives up
};

// One system of a batch, for one parity of its position buffers.
template <class M>
struct SysDesc {
    RowArgs<M> A[2];                  // the row walks' arguments; A[f].pos = the current buffer after f flips
    typename M::pos_t* pnext[2];      // the other buffer
    ListParams lp;
    StepArgs a;
    int npad, nchunk, nsc, rel, tmax;
    const int* morton_rank;
    int *cell_of, *slot_of, *order, *cell_count, *chunk_sum, *cell_start;
    unsigned long long *x, *v, *xt, *vt;
    int *idw, *idt;
    typename M::pos_t* post;
    typename M::pos_t* xref;
    uint16_t* nbr;
    int* nnb;
    int* resid;
};

// Offsets of each system's items in the batch-wide numbering (K + 1 entries
// per kind, the last the total): particles, padded cells, scan chunks, cell
// groups.
enum { BK_PART = 0, BK_CELL = 1, BK_CHUNK = 2, BK_GROUP = 3, BK_NKIND = 4 };

__device__ __forceinline__ unsigned int ld_volatile(const unsigned int* p) { return *(const volatile unsigned int*)p; }
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid-wide wait with an iteration limit.  gen is this block's count of
// completed waits.  Returns false once any block has given up.
__device__ __forceinline__ bool grid_wait(BatchCtl* ctl, unsigned int& gen)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int g = gen;
        if (atomicAdd(&ctl->count, 1u) == gridDim.x - 1) {
            ctl->count = 0u;  // nobody adds to it again before gen moves on
            __threadfence();
            atomicExch(&ctl->gen, g + 1u);
        } else {
            long long it = 0;
            while (ld_volatile(&ctl->gen) == g) {
                if (++it > ctl->wait_limit) {
                    atomicExch(&ctl->timeout, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        gen = g + 1u;
        __threadfence();
    }
    __syncthreads();
    return ld_volatile(&ctl->timeout) == 0;
}

// Largest k in [0, K) with off[k] <= w (off ascending, off[0] = 0).
__device__ __forceinline__ int batch_find(const int* off, int K, int w)
{
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Items of each system in a row walk (a block per dense cell group, or a block
// per four list entries when sparse), as offsets in shared memory.  The whole
// block calls it after the wait that ends the phase producing the lists.
template <class M, class Items>
__device__ __forceinline__ int row_offsets(const SysDesc<M>* D, int K, int* off, int* sw, Items&& items)
{
    __syncthreads();
    const int per = (K + SC_TPB - 1) / SC_TPB;
    const int b0 = min(K, (int)threadIdx.x * per), b1 = min(K, b0 + per);
    int sum = 0;
    for (int k = b0; k < b1; ++k) {
        off[k] = items(D[k]);
        sum += off[k];
    }
    int total;
    int run = block_exclusive_scan<SC_TPB>(sum, sw, total);
    for (int k = b0; k < b1; ++k) {
        const int v = off[k];
        off[k] = run;
        run += v;
    }
    if (threadIdx.x == 0) off[K] = total;
    __syncthreads();
    return total;
}

// One loop iteration (epilogue EPI) of every system of the batch.  flip is
// the number of buffer flips since the descriptors were made, mod 2.  Shared
// memory: the largest phase need of any system (smem_phase bytes), then the
// item offsets (BK_NKIND + 1 arrays of K + 1 ints).
#ifndef BATCH_MIN_BLOCKS
#define BATCH_MIN_BLOCKS 6
#endif
template <class M, int EPI>
__global__ void __launch_bounds__(SC_TPB, BATCH_MIN_BLOCKS) k_batch_iter(const SysDesc<M>* __restrict__ D, int K,
                                                       const int* __restrict__ offs, BatchCtl* ctl, int flip,
                                                       int smem_phase)
{
    // an earlier launch of this call gave up: the state is incomplete, do nothing
    if (ld_volatile(&ctl->timeout)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_n;
    __shared__ int sw[SC_TPB / 32];
    int* off = (int*)(smem + smem_phase);  // [BK_NKIND][K + 1], then the row items [K + 1]
    int* roff_items = off + BK_NKIND * (K + 1);
    for (int i = threadIdx.x; i < BK_NKIND * (K + 1); i += SC_TPB) off[i] = offs[i];
    const int* opart = off + BK_PART * (K + 1);
    const int* ocell = off + BK_CELL * (K + 1);
    const int* ochunk = off + BK_CHUNK * (K + 1);
    const int* ogroup = off + BK_GROUP * (K + 1);
    unsigned int gen = ld_volatile(&ctl->gen);
    const int nthreads = gridDim.x * SC_TPB;
    const int tid = blockIdx.x * SC_TPB + threadIdx.x;

    // ---- gate: the iteration counter, the work lists, whether a rebuild is due
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) ctl->any_due = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += SC_TPB) {
            Status* st = D[k].A[0].st;
            st->iter += 1;
            st->nwin = 0;
            st->nu = 0;
            st->ngen = 0;
            if (st->rebuild && !halted(st)) atomicExch(&ctl->any_due, 1);
        }
    }
    if (!grid_wait(ctl, gen)) return;

    if (ld_volatile(&ctl->any_due)) {
        // ---- rebuild of the systems that need one: bin, scan, scatter, sort cells, permute, build
        for (int i = tid; i < opart[K]; i += nthreads) {
            const int k = batch_find(opart, K, i);
            const SysDesc<M>& d = D[k];
            if (rebuild_on(d.A[flip].st))
                bin_item<M>(i - opart[k], d.A[flip].pos, d.A[0].g, d.morton_rank, d.cell_of, d.slot_of, d.cell_count,
                            d.A[0].st);
        }
        if (!grid_wait(ctl, gen)) return;
        for (int w = blockIdx.x; w < ochunk[K]; w += gridDim.x) {
            const int k = batch_find(ochunk, K, w);
            const SysDesc<M>& d = D[k];
            if (!rebuild_on(d.A[0].st)) continue;
            __syncthreads();
            scan_sums_chunk<SC_TPB>(w - ochunk[k], d.cell_count, d.npad, d.chunk_sum, sw);
        }
        if (!grid_wait(ctl, gen)) return;
        for (int w = blockIdx.x; w < ochunk[K]; w += gridDim.x) {
            const int k = batch_find(ochunk, K, w);
            const SysDesc<M>& d = D[k];
            Status* st = d.A[0].st;
            if (!st->rebuild || st->frozen) continue;  // raises `crowded` itself
            __syncthreads();
            scan_apply_chunk<SC_TPB>(w - ochunk[k], d.cell_count, d.npad, d.chunk_sum, d.cell_start, st, sw);
        }
        if (!grid_wait(ctl, gen)) return;
        for (int i = tid; i < opart[K]; i += nthreads) {
            const int k = batch_find(opart, K, i);
            const SysDesc<M>& d = D[k];
            if (!rebuild_on(d.A[0].st)) continue;
            const int j = i - opart[k];
            d.order[d.A[0].G.cell_start[d.cell_of[j]] + d.slot_of[j]] = j;
        }
        if (!grid_wait(ctl, gen)) return;
        for (int i = tid; i < ocell[K]; i += nthreads) {
            const int k = batch_find(ocell, K, i);
            const SysDesc<M>& d = D[k];
            if (rebuild_on(d.A[0].st)) cellsort_item(i - ocell[k], d.A[0].G.cell_start, d.order);
        }
        if (!grid_wait(ctl, gen)) return;
        for (int i = tid; i < opart[K]; i += nthreads) {
            const int k = batch_find(opart, K, i);
            const SysDesc<M>& d = D[k];
            if (rebuild_on(d.A[0].st))
                permute_item<M>(i - opart[k], d.A[0].n, d.order, d.x, d.v, d.idw, d.A[flip].pos, d.xt, d.vt, d.idt,
                                d.post);
        }
        if (!grid_wait(ctl, gen)) return;
        for (int i = tid; i < opart[K]; i += nthreads) {
            const int k = batch_find(opart, K, i);
            const SysDesc<M>& d = D[k];
            if (rebuild_on(d.A[0].st))
                copyback_item<M>(i - opart[k], d.A[0].n, d.xt, d.vt, d.idt, d.post, d.x, d.v, d.idw, d.A[flip].pos,
                                 d.xref, d.resid);
        }
        if (!grid_wait(ctl, gen)) return;
        for (int w = blockIdx.x; w < ogroup[K]; w += gridDim.x) {
            const int k = batch_find(ogroup, K, w);
            const SysDesc<M>& d = D[k];
            if (!rebuild_on(d.A[0].st)) continue;
            __syncthreads();  // the previous group is done with the shared memory
            const RowArgs<M>& A = d.A[flip];
            if constexpr (!M::fp64) {
                if (d.rel) {
                    nlist_group<M, true>(w - ogroup[k], A.g, A.pos, A.G, A.cp, d.lp, d.nbr, d.nnb, A.aux, A.st,
                                         smem);
                    continue;
                }
            }
            nlist_group<M, false>(w - ogroup[k], A.g, A.pos, A.G, A.cp, d.lp, d.nbr, d.nnb, A.aux, A.st, smem);
        }
        if (!grid_wait(ctl, gen)) return;
    }

    // ---- pass 1: close counts (and the whole soft-core forces they settle)
    for (int w = blockIdx.x; w < ogroup[K]; w += gridDim.x) {
        const int k = batch_find(ogroup, K, w);
        const RowArgs<M>& A = D[k].A[flip];
        const int b = w - ogroup[k];
        if (b == 0 && threadIdx.x == 0) A.st->rebuild = 0;
        if (halted(A.st)) continue;
        count_near_group<M>(b, A.n, A.g, A.c, A.pos, A.G, A.cp, A.aux, A.nnb, A.ds, A.sA, A.out, A.ulist, A.st, smem);
    }
    if (!grid_wait(ctl, gen)) return;

    // ---- the row walks: count, chain-rule terms, forces; each system sparse or dense on its own
    {
        const int total = row_offsets(D, K, roff_items, sw, [&](const SysDesc<M>& d) {
            const RowArgs<M>& A = d.A[flip];
            if (halted(A.st)) return 0;
            return count_rows_dense(A) ? d.nsc : (A.st->nu + SC_TPB / 32 - 1) / (SC_TPB / 32);
        });
        for (int w = blockIdx.x; w < total; w += gridDim.x) {
            const int k = batch_find(roff_items, K, w);
            const RowArgs<M>& A = D[k].A[flip];
            const int u = w - roff_items[k];
            if (count_rows_dense(A)) {
                count_rows_group<M, SC_TPB>(A, u, D[k].tmax, smem, &s_n);
            } else {
                const int e = u * (SC_TPB / 32) + (threadIdx.x >> 5);
                if (e < A.st->nu) count_rows_item(A, e);
            }
        }
    }
    if (!grid_wait(ctl, gen)) return;
    {
        const int total = row_offsets(D, K, roff_items, sw, [&](const SysDesc<M>& d) {
            const RowArgs<M>& A = d.A[flip];
            if (halted(A.st)) return 0;
            return chain_dense(A) ? d.nsc : (A.st->nwin + SC_TPB / 32 - 1) / (SC_TPB / 32);
        });
        for (int w = blockIdx.x; w < total; w += gridDim.x) {
            const int k = batch_find(roff_items, K, w);
            const RowArgs<M>& A = D[k].A[flip];
            const int u = w - roff_items[k];
            if (chain_dense(A)) {
                chain_group<M, SC_TPB>(A, u, D[k].tmax, smem, &s_n);
            } else {
                const int e = u * (SC_TPB / 32) + (threadIdx.x >> 5);
                if (e < A.st->nwin) chain_item(A, e);
            }
        }
    }
    if (!grid_wait(ctl, gen)) return;
    {
        const int total = row_offsets(D, K, roff_items, sw, [&](const SysDesc<M>& d) {
            const RowArgs<M>& A = d.A[flip];
            if (halted(A.st)) return 0;
            return force_dense(A) ? d.nsc : (A.st->ngen + SC_TPB / 32 - 1) / (SC_TPB / 32);
        });
        for (int w = blockIdx.x; w < total; w += gridDim.x) {
            const int k = batch_find(roff_items, K, w);
            const RowArgs<M>& A = D[k].A[flip];
            const int u = w - roff_items[k];
            if (force_dense(A)) {
                force_group<M, SC_TPB>(A, u, D[k].tmax, smem, &s_n);
            } else {
                const int e = u * (SC_TPB / 32) + (threadIdx.x >> 5);
                if (e < A.st->ngen) force_item(A, e);
            }
        }
    }
    if (!grid_wait(ctl, gen)) return;

    // ---- the update of every particle
    for (int i = tid; i < opart[K]; i += nthreads) {
        const int k = batch_find(opart, K, i);
        const SysDesc<M>& d = D[k];
        const RowArgs<M>& A = d.A[flip];
        if (!halted(A.st))
            step_item<M, EPI>(i - opart[k], A.n, A.g, A.aux, A.id, d.pnext[flip], d.xref, d.a, A.st);
    }
}

}  // namespace vbc
