// sortscan.cuh -- device-wide scans and stream compactions driven by
// functors (over any values, and over one flag byte per element), the run
// tiles of a batch's sorted node-view entries, and a stable LSD radix sort
// of (key, u32 value) pairs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "prims.cuh"

namespace tw {

// ---------------------------------------------------------------------------
// Two-level scan / compaction.
// Op supplies  __device__ uint64_t value(int64_t i) const
//              __device__ void emit(int64_t i, uint64_t v, uint64_t excl) const
// Phase 1 sums value() over each block's contiguous range, phase 2 scans the
// block sums (one block), phase 3 rescans each range and calls emit() with
// the exclusive prefix.  value() is evaluated twice per element.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;
constexpr int SCAN_MAX_BLOCKS = 2048;

template <class Op, int ITEMS>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(Op op, int64_t n, int64_t per_blk,
                                                              uint64_t *partials)
{
    __shared__ uint64_t wt[32];
    const int64_t b0 = (int64_t)blockIdx.x * per_blk;
    const int64_t b1 = min(n, b0 + per_blk);
    uint64_t s = 0;
    // ITEMS values per thread per chunk, evaluated together (their
    // loads are independent), in the striped order the emit pass reads
    for (int64_t c = b0; c < b1; c += (SCAN_THREADS * ITEMS)) {
        uint64_t v[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int64_t i = c + k * SCAN_THREADS + threadIdx.x;
            v[k] = (i < b1) ? op.value(i) : 0;
        }
#pragma unroll
        for (int k = 0; k < ITEMS; k++) s += v[k];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += wt[w];
        partials[blockIdx.x] = t;
    }
}

// Exclusive scan of partials[0..nb) in place (one block of 1024 threads);
// partials[nb] receives the total.
__global__ void k_scan_partials(uint64_t *partials, int nb);

// Each chunk of SCAN_THREADS * ITEMS elements is read and written in striped
// order (element c + k*THREADS + thread, so a warp touches consecutive
// elements) and staged through shared memory, where each thread scans ITEMS
// consecutive values.
// Shared-memory slot of staged element j: one pad slot per 16 (a thread's
// ITEMS consecutive 8-byte values sit 64 B apart from the next thread's at
// ITEMS = 8, which without the pad maps a half-warp onto two banks).
__device__ __forceinline__ int scan_slot(int j) { return j + (j >> 4); }

template <class Op, int ITEMS>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_emit(Op op, int64_t n, int64_t per_blk,
                                                            const uint64_t *partials)
{
    __shared__ uint64_t wt[33];
    __shared__ uint64_t sv[(SCAN_THREADS * ITEMS) + (SCAN_THREADS * ITEMS) / 16];  // values, then exclusive prefixes
    const int64_t b0 = (int64_t)blockIdx.x * per_blk;
    const int64_t b1 = min(n, b0 + per_blk);
    uint64_t carry = partials[blockIdx.x];
    for (int64_t c = b0; c < b1; c += (SCAN_THREADS * ITEMS)) {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int j = k * SCAN_THREADS + threadIdx.x;
            const int64_t i = c + j;
            sv[scan_slot(j)] = (i < b1) ? op.value(i) : 0;
        }
        __syncthreads();
        uint64_t v[ITEMS];
        uint64_t s = 0;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            v[k] = sv[scan_slot(threadIdx.x * ITEMS + k)];
            s += v[k];
        }
        uint64_t tot;
        uint64_t ex = block_excl_scan<uint64_t>(s, wt, tot);  // synchronises
        ex += carry;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            sv[scan_slot(threadIdx.x * ITEMS + k)] = ex;
            ex += v[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int j = k * SCAN_THREADS + threadIdx.x;
            const int64_t i = c + j;
            if (i < b1) {
                const uint64_t e = sv[scan_slot(j)];
                const uint64_t nx = (j + 1 < (SCAN_THREADS * ITEMS)) ? sv[scan_slot(j + 1)] : carry + tot;
                op.emit(i, nx - e, e);
            }
        }
        carry += tot;
        __syncthreads();
    }
}

// Host driver.  partials must hold SCAN_MAX_BLOCKS + 1 entries; the total
// ends in partials[nb] where nb is returned.  ITEMS: values per thread per
// chunk; 1 for an op whose value() is a chain of dependent loads over a
// modest n (more blocks in flight instead of more values per thread).
template <class Op, int ITEMS = SCAN_ITEMS>
int scan_launch(const Op &op, int64_t n, uint64_t *partials, cudaStream_t st)
{
    if (n <= 0) {
        cudaMemsetAsync(partials, 0, sizeof(uint64_t), st);
        return 0;
    }
    constexpr int64_t CHUNK = (int64_t)SCAN_THREADS * ITEMS;
    int64_t nb = (n + CHUNK - 1) / CHUNK;
    if (nb > SCAN_MAX_BLOCKS) nb = SCAN_MAX_BLOCKS;
    int64_t per = (n + nb - 1) / nb;
    per = (per + CHUNK - 1) / CHUNK * CHUNK;
    nb = (n + per - 1) / per;
    k_scan_reduce<Op, ITEMS><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(op, n, per, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, (int)nb);
    k_scan_emit<Op, ITEMS><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(op, n, per, partials);
    return (int)nb;
}

// ---------------------------------------------------------------------------
// Two-level scans over one flag byte per element.  Each thread takes 16
// consecutive bytes with one 16-byte load and evaluates their values in
// registers (bit masks of the bytes), a block scans the thread sums, and the
// op writes its outputs from registers.  Elements are addressed through a
// virtual index u = i + a from a 16-byte aligned base (a = the flags'
// misalignment), so every load is aligned; the bytes outside [a, a + n) are
// masked, and the allocation must extend to the next 16-byte boundary after
// the last element.  Op supplies
//   __host__ __device__ int64_t tiles() const;           // tiles of BSCAN_TILE virtual elements
//   __device__ uint4 load(int64_t u0) const;             // the 16 bytes at virtual index u0
//   __device__ uint64_t sum16(uint4 w, int64_t u0) const;  // sum of their values
//   __device__ void emit16(uint4 w, int64_t u0, uint64_t ex, uint64_t tile_ex, uint64_t tile_tot,
//                          Stage &sm) const;             // ex: exclusive prefix of u0's first element
//   struct Stage;                                        // the op's shared memory per block
// emit16 is called by every thread of the block (it may synchronise).
// ---------------------------------------------------------------------------
constexpr int BSCAN_THREADS = 256;
constexpr int BSCAN_TILE = BSCAN_THREADS * 16;

// Bit k of the result is bit b of byte k of w.  (((x >> b) & 0x01010101) *
// 0x10204080) >> 28 gathers the bit of byte q of x into bit q: the four
// products that land in bits 28-31 are the wanted ones, and the others fall
// on distinct lower bits, so no carry reaches them.
__device__ __forceinline__ uint32_t byte_bits16(uint4 w, int b)
{
    const uint32_t m = 0x01010101u;
    return ((((w.x >> b) & m) * 0x10204080u) >> 28) | (((((w.y >> b) & m) * 0x10204080u) >> 28) << 4) |
           (((((w.z >> b) & m) * 0x10204080u) >> 28) << 8) | (((((w.w >> b) & m) * 0x10204080u) >> 28) << 12);
}

// Mask of the 16 virtual elements from u0 that fall in [a, a + n).
__device__ __forceinline__ uint32_t valid16(int64_t u0, int64_t a, int64_t n)
{
    const int64_t lo = a - u0, hi = a + n - u0;
    const uint32_t hm = hi >= 16 ? 0xffffu : (hi <= 0 ? 0u : (1u << hi) - 1u);
    const uint32_t lm = lo <= 0 ? 0u : (lo >= 16 ? 0xffffu : (1u << lo) - 1u);
    return hm & ~lm;
}

template <class Op>
__global__ void __launch_bounds__(BSCAN_THREADS) k_bscan_reduce(Op op, int64_t per, uint64_t *partials)
{
    __shared__ uint64_t wt[32];
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(op.tiles(), t0 + per);
    uint64_t s = 0;
    for (int64_t t = t0; t < t1; t += 2) {  // two loads in flight per thread
        const int64_t u0 = t * BSCAN_TILE + 16 * threadIdx.x, u1 = u0 + BSCAN_TILE;
        const uint4 w0 = op.load(u0);
        const uint4 w1 = t + 1 < t1 ? op.load(u1) : make_uint4(0, 0, 0, 0);
        s += op.sum16(w0, u0);
        if (t + 1 < t1) s += op.sum16(w1, u1);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += wt[w];
        partials[blockIdx.x] = t;
    }
}

template <class Op>
__global__ void __launch_bounds__(BSCAN_THREADS) k_bscan_emit(Op op, int64_t per, const uint64_t *partials)
{
    __shared__ uint64_t wt[33];
    __shared__ typename Op::Stage sm;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(op.tiles(), t0 + per);
    uint64_t carry = partials[blockIdx.x];
    uint4 w = t0 < t1 ? op.load(t0 * BSCAN_TILE + 16 * threadIdx.x) : make_uint4(0, 0, 0, 0);
    for (int64_t t = t0; t < t1; t++) {
        const int64_t u0 = t * BSCAN_TILE + 16 * threadIdx.x;
        // the next tile's bytes in flight while this one is scanned
        const uint4 wn = t + 1 < t1 ? op.load(u0 + BSCAN_TILE) : make_uint4(0, 0, 0, 0);
        uint64_t tot;
        const uint64_t ex = block_excl_scan<uint64_t>(op.sum16(w, u0), wt, tot);  // synchronises
        op.emit16(w, u0, carry + ex, carry, tot, sm);
        carry += tot;
        w = wn;
    }
}

// Host driver, as scan_launch: partials must hold SCAN_MAX_BLOCKS + 1
// entries; the total ends in partials[nb] where nb is returned.
template <class Op>
int bscan_launch(const Op &op, uint64_t *partials, cudaStream_t st)
{
    const int64_t tiles = op.tiles();
    if (tiles <= 0) {
        cudaMemsetAsync(partials, 0, sizeof(uint64_t), st);
        return 0;
    }
    int64_t nb = tiles < SCAN_MAX_BLOCKS ? tiles : SCAN_MAX_BLOCKS;
    const int64_t per = (tiles + nb - 1) / nb;
    nb = (tiles + per - 1) / per;
    k_bscan_reduce<Op><<<(unsigned)nb, BSCAN_THREADS, 0, st>>>(op, per, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, (int)nb);
    k_bscan_emit<Op><<<(unsigned)nb, BSCAN_THREADS, 0, st>>>(op, per, partials);
    return (int)nb;
}

// Runs of a batch's sorted entries, one block per tile of BSCAN_TILE
// entries.  From the entries' flag bytes (bit 0: a run starts, bit 1: a group
// starts) and the tile's prefix (runs and groups before the tile, high and
// low 32 bits), every entry's run and the batch's groups before it, for
// loops over the tile's entries in any order.  Replaces two int32 arrays per
// entry written by the run scan and read back by its consumers.
struct RunTile {
    uint32_t rm[BSCAN_THREADS], gm[BSCAN_THREADS];  // each thread's 16 entries: run / group start masks
    uint64_t ex[BSCAN_THREADS];                     // prefix before each thread's first entry
    uint64_t wt[33];
};

struct RunAt {
    int32_t r;  // the entry's run
    int32_t g;  // groups of the batch before it
    bool rs, gs;  // it starts a run / a group
};

// Every thread of the block calls it (it synchronises).
__device__ __forceinline__ void run_tile_load(RunTile &sm, const uint8_t *__restrict__ flags, int64_t n, int64_t t,
                                              uint64_t tile_prefix)
{
    const int64_t u0 = t * BSCAN_TILE + 16 * threadIdx.x;
    const uint4 w = u0 < n ? __ldg(reinterpret_cast<const uint4 *>(flags + u0)) : make_uint4(0, 0, 0, 0);
    const uint32_t v = valid16(u0, 0, n);
    const uint32_t rm = byte_bits16(w, 0) & v, gm = byte_bits16(w, 1) & v;
    uint64_t tot;
    const uint64_t ex = block_excl_scan<uint64_t>(((uint64_t)__popc(rm) << 32) | (uint64_t)__popc(gm), sm.wt, tot);
    sm.rm[threadIdx.x] = rm;
    sm.gm[threadIdx.x] = gm;
    sm.ex[threadIdx.x] = tile_prefix + ex;
    __syncthreads();
}

// Entry j of the tile (0 <= j < BSCAN_TILE).
__device__ __forceinline__ RunAt run_tile_at(const RunTile &sm, int j)
{
    const int o = j >> 4, q = j & 15;
    const uint32_t below = (1u << q) - 1u, rm = sm.rm[o], gm = sm.gm[o];
    const uint64_t ex = sm.ex[o];
    RunAt a;
    a.rs = (rm >> q) & 1u;
    a.gs = (gm >> q) & 1u;
    a.r = (int32_t)((uint32_t)(ex >> 32) + (uint32_t)__popc(rm & below) + (a.rs ? 0u : 0xffffffffu));
    a.g = (int32_t)((uint32_t)ex + (uint32_t)__popc(gm & below));
    return a;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs, 8-bit digits.
// A Loader supplies the input of the first pass:
//   __device__ K key(int64_t i) const;  __device__ uint32_t val(int64_t i) const;
// later passes read the previous pass's output.  Each block owns a
// contiguous range of tiles; within a tile, warps rank their elements with
// match_any, the block orders them by digit in shared memory and writes out
// runs of equal digits to consecutive addresses.
// ---------------------------------------------------------------------------
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SORT_MAX_BLOCKS = 4096;  // one 2048-key tile per block up to 8M keys (part[] holds <= 256 chunks)

// A loader whose key is computed (not read) may keep it: the histogram pass
// calls note(i, key) for each element, and the first scatter pass can then
// read the kept keys (radix_sort_launch's second loader).
template <class L, class = void>
struct loader_notes : std::false_type {};
template <class L>
struct loader_notes<L, std::void_t<decltype(std::declval<const L &>().note(int64_t(0), uint32_t(0)))>>
    : std::true_type {};

template <typename K>
struct ArrayLoader {
    const K *k;
    const uint32_t *v;
    __device__ __forceinline__ K key(int64_t i) const { return k[i]; }
    __device__ __forceinline__ uint32_t val(int64_t i) const { return v[i]; }
};

template <typename K, class L>
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(L ld, int64_t n, int64_t per_blk,
                                                             int shift, uint32_t *hist, int nblk)
{
    __shared__ uint32_t h[SORT_WARPS][RADIX];
    for (int i = threadIdx.x; i < SORT_WARPS * RADIX; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b0 = (int64_t)blockIdx.x * per_blk;
    const int64_t b1 = min(n, b0 + per_blk);
    constexpr int U = 4;  // keys per thread loaded together (independent loads in flight)
    for (int64_t base = b0; base < b1; base += (int64_t)U * blockDim.x) {
        uint32_t d[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t i = base + u * blockDim.x + threadIdx.x;
            d[u] = 0xffffu;
            if (i < b1) {
                const K k = ld.key(i);
                if constexpr (loader_notes<L>::value) ld.note(i, (uint32_t)k);
                d[u] = (uint32_t)((k >> shift) & (RADIX - 1));
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t peers = __match_any_sync(0xffffffffu, d[u]);
            const int leader = __ffs(peers) - 1;
            if (d[u] != 0xffffu && lane == leader) h[w][d[u]] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < SORT_WARPS; k++) s += h[k][d];
        hist[(int64_t)d * nblk + blockIdx.x] = s;
    }
}

// Exclusive scan of the digit histogram, in two kernels: every 1024-thread
// block scans a chunk of HSCAN_CHUNK counts in place and leaves the chunk
// total in part[]; one block then scans part[].  The scatter adds part[] of
// the chunk to each offset it reads.  part[] follows the histogram (the
// histogram buffer holds SORT_HIST_WORDS u32).
constexpr int HSCAN_CHUNK = 4096;
constexpr int64_t SORT_HIST_WORDS = (int64_t)RADIX * SORT_MAX_BLOCKS + 1 + 2 * 128;

static __global__ void __launch_bounds__(1024) k_hscan_local(uint32_t *a, int64_t n, uint32_t *part)
{
    __shared__ uint32_t sh[33];
    const int64_t c0 = (int64_t)blockIdx.x * HSCAN_CHUNK + (int64_t)threadIdx.x * 4;
    uint32_t v[4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = c0 + k < n ? a[c0 + k] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<uint32_t>(s, sh, tot);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (c0 + k < n) a[c0 + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(1024) k_hscan_part(uint32_t *part, int nb)
{
    __shared__ uint32_t sh[33];
    const uint32_t v = (int)threadIdx.x < nb ? part[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan<uint32_t>(v, sh, tot);
    if ((int)threadIdx.x < nb) part[threadIdx.x] = ex;
}

template <typename K, class L>
__global__ void __launch_bounds__(SORT_THREADS, sizeof(K) == 4 ? 5 : 3) k_radix_scatter(L ld, K *kout, uint32_t *vout,
                                                                int64_t n, int64_t per_blk, int shift,
                                                                const uint32_t *offs, const uint32_t *part,
                                                                int nblk)
{
    __shared__ uint32_t run_off[RADIX];
    __shared__ uint32_t wcnt[SORT_WARPS][RADIX];
    __shared__ uint32_t dstart[RADIX];
    __shared__ uint32_t dcnt[RADIX];
    __shared__ K sk[SORT_TILE];
    __shared__ uint32_t sv[SORT_TILE];
    __shared__ uint32_t wt[33];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t b0 = (int64_t)blockIdx.x * per_blk;
    const int64_t b1 = min(n, b0 + per_blk);
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
        const int64_t x = (int64_t)d * nblk + blockIdx.x;
        run_off[d] = offs[x] + part[x / HSCAN_CHUNK];
    }

    for (int64_t t0 = b0; t0 < b1; t0 += SORT_TILE) {
        for (int i = threadIdx.x; i < SORT_WARPS * RADIX; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        K kk[SORT_ITEMS];
        uint32_t vv[SORT_ITEMS];
        uint32_t dd[SORT_ITEMS];
        uint32_t rk[SORT_ITEMS];
        const int64_t chunk = t0 + (int64_t)w * 32 * SORT_ITEMS;
        // all SORT_ITEMS loads in flight before the ranking (whose warp
        // barriers would otherwise hold each load until the previous rank)
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; r++) {
            const int64_t i = chunk + r * 32 + lane;
            if (i < b1) {
                kk[r] = ld.key(i);
                vv[r] = ld.val(i);
            } else {
                kk[r] = K(0);
                vv[r] = 0;
            }
        }
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; r++) {
            const bool ok = chunk + r * 32 + lane < b1;
            dd[r] = ok ? (uint32_t)((kk[r] >> shift) & (RADIX - 1)) : 0xffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, dd[r]);
            const uint32_t pre = ok ? wcnt[w][dd[r]] : 0u;
            __syncwarp();
            if (ok && (peers & lt) == 0) wcnt[w][dd[r]] = pre + __popc(peers);
            __syncwarp();
            rk[r] = pre + __popc(peers & lt);
        }
        __syncthreads();
        // per digit: exclusive prefix over warps and the tile count
        for (int d = threadIdx.x; d < RADIX; d += blockDim.x) {
            uint32_t s = 0;
#pragma unroll
            for (int k = 0; k < SORT_WARPS; k++) {
                const uint32_t c = wcnt[k][d];
                wcnt[k][d] = s;
                s += c;
            }
            dcnt[d] = s;
        }
        __syncthreads();
        {
            // exclusive scan of dcnt over digits (RADIX == blockDim)
            uint32_t tot;
            const uint32_t c = (threadIdx.x < RADIX) ? dcnt[threadIdx.x] : 0u;
            const uint32_t ex = block_excl_scan<uint32_t>(c, wt, tot);
            if (threadIdx.x < RADIX) dstart[threadIdx.x] = ex;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; r++) {
            if (dd[r] != 0xffffu) {
                const uint32_t p = dstart[dd[r]] + wcnt[w][dd[r]] + rk[r];
                sk[p] = kk[r];
                sv[p] = vv[r];
            }
        }
        __syncthreads();
        const int tile_n = (int)min((int64_t)SORT_TILE, b1 - t0);
        for (int j = threadIdx.x; j < tile_n; j += blockDim.x) {
            const K k = sk[j];
            const uint32_t d = (uint32_t)((k >> shift) & (RADIX - 1));
            const uint32_t g = run_off[d] + (uint32_t)j - dstart[d];
            kout[g] = k;
            vout[g] = sv[j];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += blockDim.x) run_off[d] += dcnt[d];
        __syncthreads();
    }
}

// Sorts n pairs by the low `bits` bits of the key.  The loader provides the
// input (it must not read k[0] / v[0], which the first pass writes);
// k[0..1], v[0..1] are double buffers of n elements.  Returns the
// buffer index (0 or 1) holding the result, or -1 when no pass ran (the
// input already has all keys equal in those bits; the caller then uses the
// loader's data as is).  hist needs RADIX * nblocks + 1 + 2 * 128 u32 (at most
// SORT_HIST_WORDS).
template <typename K, class L, class L0>
int radix_sort_launch(const L &ld, const L0 &ld0, int64_t n, int bits, K *k[2], uint32_t *v[2], uint32_t *hist,
                      cudaStream_t st, int *launches);

template <typename K, class L>
int radix_sort_launch(const L &ld, int64_t n, int bits, K *k[2], uint32_t *v[2], uint32_t *hist,
                      cudaStream_t st, int *launches)
{
    return radix_sort_launch<K, L, L>(ld, ld, n, bits, k, v, hist, st, launches);
}

// The same with the first scatter pass reading its input through ld0 (the
// keys the first histogram pass noted, for instance).
template <typename K, class L, class L0>
int radix_sort_launch(const L &ld, const L0 &ld0, int64_t n, int bits, K *k[2], uint32_t *v[2], uint32_t *hist,
                      cudaStream_t st, int *launches)
{
    if (n <= 0 || bits <= 0) return -1;
    int64_t nb = (n + SORT_TILE - 1) / SORT_TILE;
    if (nb > SORT_MAX_BLOCKS) nb = SORT_MAX_BLOCKS;
    int64_t per = (n + nb - 1) / nb;
    per = (per + SORT_TILE - 1) / SORT_TILE * SORT_TILE;
    nb = (n + per - 1) / per;
    const int passes = (bits + RADIX_BITS - 1) / RADIX_BITS;
    const int64_t hn = (int64_t)RADIX * nb;
    const int hchunks = (int)((hn + HSCAN_CHUNK - 1) / HSCAN_CHUNK);
    uint32_t *part = hist + hn + 1;
    int cur = -1;
    for (int p = 0; p < passes; p++) {
        const int shift = p * RADIX_BITS;
        const int out = (cur == 0) ? 1 : 0;
        if (p == 0) {
            k_radix_hist<K, L><<<(unsigned)nb, SORT_THREADS, 0, st>>>(ld, n, per, shift, hist, (int)nb);
            k_hscan_local<<<hchunks, 1024, 0, st>>>(hist, hn, part);
            k_hscan_part<<<1, 1024, 0, st>>>(part, hchunks);
            k_radix_scatter<K, L0><<<(unsigned)nb, SORT_THREADS, 0, st>>>(ld0, k[out], v[out], n, per, shift,
                                                                           hist, part, (int)nb);
        } else {
            ArrayLoader<K> al{k[cur], v[cur]};
            k_radix_hist<K, ArrayLoader<K>><<<(unsigned)nb, SORT_THREADS, 0, st>>>(al, n, per, shift, hist,
                                                                                  (int)nb);
            k_hscan_local<<<hchunks, 1024, 0, st>>>(hist, hn, part);
            k_hscan_part<<<1, 1024, 0, st>>>(part, hchunks);
            k_radix_scatter<K, ArrayLoader<K>><<<(unsigned)nb, SORT_THREADS, 0, st>>>(
                al, k[out], v[out], n, per, shift, hist, part, (int)nb);
        }
        if (launches) *launches += 4;
        cur = out;
    }
    return cur;
}

}  // namespace tw
