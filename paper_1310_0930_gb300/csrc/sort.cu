// sort.cu -- periodic counting sort of the particles by tile.
//
// The GPU counterpart of the paper's particle migration between nodes after
// the push (Sec. 3): particles that moved are regrouped with the tile that
// now owns them, dead slots (absorbed particles) are dropped, and the tail
// of freshly injected plasma is merged.  The key of a particle
// is (tile, sub-bucket).  By default the sub-bucket is the particle's row of
// cells along x inside the tile (its y and z cell in the tile), so a tile's
// particles come out grouped by row: the particles a warp pushes together
// then lie in one or two rows, and their field-tile loads share addresses
// (broadcast) or fall in adjacent banks.  Optionally (pic_tuning.sort_sub)
// the sub-bucket of slot i is i mod nsub, which interleaves the particles of
// a cell over the tile's range.
// Steps, per run:
//   1. zero the key counters;
//   2. histogram of keys, aggregated per warp (match on the key) and per CTA
//      (a shared-memory key table over a chunk of kSortChunk slots), so that
//      the global counters see a few atomics per chunk; where each thread's
//      four consecutive slots share one key (a chunk still in sorted order)
//      the warp counts them as one item of weight four;
//   3. exclusive scan of the counters in blocks of kScanChunk keys (block
//      sums, an exclusive scan of the block sums, then each block adds its
//      prefix); the counters become the scatter cursors and tile_off[t] the
//      offset of key (t, 0);
//   4. scatter every live particle into the alternate buffer at
//      offset[key] + rank: ranks within the chunk come from the CTA's key
//      table (weight-four items as in the count, ranked so that the lanes
//      of one store instruction write consecutive slots), and one cursor
//      atomic per (chunk, key) reserves the range;
//   5. flip the buffer and set the sorted count.
// Order within a key is not stable (cursor atomics); nothing downstream
// depends on it.
#include "common.cuh"
#include "internal.h"

namespace pic {

namespace {

__device__ __forceinline__ int seg_run(const Seg &s, int b)
{
    int lo = 0, hi = s.nruns - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s.start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Grid-stride walk over the chunks of a particle segment: the next chunk of
// this CTA at or after chunk `from` (chunks b with b = blockIdx.x mod
// gridDim.x), used to step over a run that does not sort this step.
__device__ __forceinline__ int next_own_chunk(int from)
{
    const int g = (int)gridDim.x, r = (from - (int)blockIdx.x) % g;
    return r == 0 ? from : from + (g - r);
}

// What the tile key of a packed cell depends on, held in registers.
struct KeyCtx {
    int b0, b1, m0, m1, t0, t1, t2, nt0, nt1, dim, open_last, origin, nl, lo, hi, nsub, rows;
    long long n_total;
};

__device__ __forceinline__ KeyCtx key_ctx(const Run &r, const RunState &s)
{
    KeyCtx k;
    k.b0 = r.bits[0];
    k.b1 = r.bits[1];
    k.m0 = (1 << r.bits[0]) - 1;
    k.m1 = (1 << r.bits[1]) - 1;
    k.t0 = r.tlog[0];
    k.t1 = r.tlog[1];
    k.t2 = r.tlog[2];
    k.nt0 = r.nt[0];
    k.nt1 = r.nt[1];
    k.dim = r.dim;
    k.open_last = r.open_last;
    k.origin = s.origin;
    k.nl = r.n[r.dim - 1];
    k.lo = r.margin;
    k.hi = r.n[r.dim - 1] - r.margin;
    k.n_total = s.n_total;
    k.nsub = r.nsub;
    k.rows = r.sort_rows;
    return k;
}

// (tile, sub-bucket) key of slot i holding packed cell c: the cell's row
// (y + ty z, cells within the tile) or the slot's interleave class
__device__ __forceinline__ int sub_key(const KeyCtx &k, int tile, long long i, int32_t c)
{
    if (tile < 0) return -1;
    if (!k.rows) return tile * k.nsub + (int)(i & (k.nsub - 1));
    const int y = (c >> k.b0) & k.m1 & ((1 << k.t1) - 1);
    const int z = k.dim == 3 ? (c >> (k.b0 + k.b1)) & ((1 << k.t2) - 1) : 0;
    return tile * k.nsub + y + (z << k.t1);
}

// tile key of a packed cell, or -1 for a dead slot / a particle outside the
// kept part of the window
__device__ __forceinline__ int key_of_cell(const KeyCtx &k, int32_t c)
{
    if (c < 0) return -1;
    const int cx = c & k.m0, cy = (c >> k.b0) & k.m1, cz = k.dim == 3 ? (c >> (k.b0 + k.b1)) : 0;
    if (k.open_last) {
        int pl = (k.dim == 3 ? cz : cy) - k.origin;
        pl = pl < 0 ? pl + k.nl : pl;
        if (pl < k.lo || pl >= k.hi) return -1;
    }
    return (cx >> k.t0) + k.nt0 * ((cy >> k.t1) + k.nt1 * (k.dim == 3 ? (cz >> k.t2) : 0));
}

// Whether each run sorts this step: when the host asks (force), or, under
// the adaptive policy, when max_interval steps have passed since the last
// sort or particles that strayed beyond their tiles' staged regions add up
// to n_total / kSortSlowDiv particle-steps since then.  A stray takes the
// slow path (global gather and global atomics) and stalls the other lanes of
// its warp meanwhile: a fraction of a percent of strays costs the push more
// than a sort, so the threshold is low.  The unsorted tail of particles
// injected by the moving window is not counted as strays (it is pushed by
// CTAs of its own); a run also sorts once its tail holds n_total /
// kSortTailDiv particles (tail particles take the slow path).
// The kernels of the sort below skip the runs that do not sort.
__global__ void sort_decide_kernel(const Run *__restrict__ runs, int nruns, int force, int max_interval,
                                   int adaptive)
{
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= nruns) return;
    RunState &s = *runs[ri].state;
    bool go = force != 0;
    if (adaptive) {
        const unsigned long long n = s.n_total > 0 ? (unsigned long long)s.n_total : 0ull;
        const unsigned long long tail = s.n_total > s.n_sorted ? (unsigned long long)(s.n_total - s.n_sorted) : 0ull;
        go = go || s.since_sort >= max_interval || (s.slow_acc > 0 && s.slow_acc * kSortSlowDiv >= n) ||
             tail * kSortTailDiv >= n;
    }
    s.do_sort = go ? 1 : 0;
    if (go) {
        s.since_sort = 0;
        s.slow_acc = 0;
        s.sorts += 1;
    }
}

__global__ void sort_zero_kernel(const Run *__restrict__ runs, int nruns)
{
    const int ri = blockIdx.y;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    if (!r.state->do_sort) return;
    const long long nk = (long long)r.ntiles * r.nsub;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nk; t += (long long)gridDim.x * blockDim.x)
        r.tile_cnt[t] = 0;
}

// Lanes of this warp holding the same key; a warp whose 32 keys agree (the
// common case: particles are still grouped by tile) skips the match.
__device__ __forceinline__ unsigned key_peers(int key)
{
    const int k0 = __shfl_sync(0xffffffffu, key, 0);
    if (__all_sync(0xffffffffu, key == k0)) return 0xffffffffu;
    return __match_any_sync(0xffffffffu, key);
}

// Per-CTA table of the keys seen in one chunk (open addressing with a
// bounded probe).  A key that finds no slot returns -1 and its warp falls
// back to a direct global atomic.
struct KeyTable {
    int key[kSortHash];
    int cnt[kSortHash];
    int base[kSortHash];
};

__device__ __forceinline__ void table_init(KeyTable &t)
{
    for (int e = threadIdx.x; e < kSortHash; e += blockDim.x) {
        t.key[e] = -1;
        t.cnt[e] = 0;
    }
}

__device__ __forceinline__ int table_slot(KeyTable &t, int key)
{
    unsigned h = ((unsigned)key * 2654435761u) >> (32 - kSortHashLog);
#pragma unroll 1
    for (int p = 0; p < kSortProbe; ++p) {
        const int e = (int)((h + p) & (kSortHash - 1));
        const int prev = atomicCAS(&t.key[e], -1, key);
        if (prev == -1 || prev == key) return e;
    }
    return -1;
}

// Slot of item j (0 .. kSortItems-1) of this thread in the chunk at i0: two
// groups of four consecutive slots, so that each thread loads its particles
// with 16-byte vector accesses.
__device__ __forceinline__ long long item_slot(long long i0, int j)
{
    return i0 + (j >> 2) * (kSortChunk / 2) + 4 * threadIdx.x + (j & 3);
}

// Four consecutive 32-bit values at p + s0 (valid ones only past n).
template <class T, class T4>
__device__ __forceinline__ void load4(const T *p, long long s0, long long n, T *out)
{
    if (s0 + 3 < n) {
        const T4 v = *reinterpret_cast<const T4 *>(p + s0);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = s0 + q < n ? p[s0 + q] : T(0);
    }
}

// The four cells of slots s0 .. s0+3; dead (-1) past n.
__device__ __forceinline__ void load_cells4(const int32_t *cell, long long s0, long long n, int32_t *out)
{
    load4<int32_t, int4>(cell, s0, n, out);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = s0 + q < n ? out[q] : -1;
}

// Tile histogram: each CTA counts a chunk of kSortChunk slots in shared
// memory (one shared atomic per warp and key), then adds its per-key totals
// to the global counters: a handful of global atomics per chunk.  All the
// chunk's cells are loaded before the first use, for memory parallelism.
__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(const Run *__restrict__ runs, Seg seg)
{
    __shared__ KeyTable t;
    for (int b = blockIdx.x; b < seg.nblocks; b += gridDim.x) {  // (CTA-uniform control flow)
        const int ri = seg_run(seg, b);
        const Run &r = runs[ri];
        if (!r.state->do_sort) {  // the run does not sort this step: skip its chunks
            b = next_own_chunk(seg.start[ri + 1]) - (int)gridDim.x;
            continue;
        }
        const KeyCtx kc = key_ctx(r, *r.state);
        const long long i0 = (long long)(b - seg.start[ri]) * kSortChunk;
        if (i0 >= kc.n_total) continue;
        const int32_t *cells = r.P[r.state->buf].cell;
        int32_t cell[kSortItems];
#pragma unroll
        for (int g = 0; g < kSortItems / 4; ++g) load_cells4(cells, item_slot(i0, 4 * g), kc.n_total, cell + 4 * g);
        table_init(t);
        __syncthreads();
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int g = 0; g < kSortItems / 4; ++g) {
            int key[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                key[q] = sub_key(kc, key_of_cell(kc, cell[4 * g + q]), item_slot(i0, 4 * g + q), cell[4 * g + q]);
            // (a sorted chunk: each thread's four consecutive slots mostly
            // share a key, and a warp counts them as one item of weight 4)
            const int nq = __all_sync(0xffffffffu, key[0] == key[1] && key[0] == key[2] && key[0] == key[3]) ? 1 : 4;
            for (int q = 0; q < nq; ++q) {
                const int kq = key[q];
                const unsigned peers = key_peers(kq);
                if (kq >= 0 && lane == __ffs(peers) - 1) {
                    const int e = table_slot(t, kq);
                    const int c = (5 - nq) * __popc(peers);
                    if (e >= 0) atomicAdd(&t.cnt[e], c);
                    else atomicAdd(&r.tile_cnt[kq], c);
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kSortHash; e += blockDim.x)
            if (t.key[e] >= 0 && t.cnt[e] > 0) atomicAdd(&r.tile_cnt[t.key[e]], t.cnt[e]);
        __syncthreads();  // (the next chunk re-initialises the table)
    }
}

// Exclusive scan of the key counters, pass 1: block b of a run scans its
// kScanChunk keys in place (exclusive, block-local) and stores its total.
// Thread t owns kScanItems consecutive keys.
__global__ void __launch_bounds__(kScanThreads) sort_scan_local_kernel(const Run *__restrict__ runs, Seg seg,
                                                                       int *__restrict__ sums)
{
    __shared__ int warp_tot[kScanThreads / 32];
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    if (!r.state->do_sort) return;  // CTA-uniform
    const long long nk = (long long)r.ntiles * r.nsub;
    const long long k0 = (long long)(blockIdx.x - seg.start[ri]) * kScanChunk + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int tot = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = k0 + q < nk ? r.tile_cnt[k0 + q] : 0;
        tot += v[q];
    }
    // block exclusive scan of the per-thread totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        before += w < wid ? warp_tot[w] : 0;
        all += warp_tot[w];
    }
    int run = before + inc - tot;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (k0 + q < nk) r.tile_cnt[k0 + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = all;
}

// Pass 2: one CTA per run scans the run's block totals in place (exclusive)
// and sets tile_off[ntiles] = the run's total.
__global__ void __launch_bounds__(kScanThreads) sort_scan_sums_kernel(const Run *__restrict__ runs, Seg seg,
                                                                      int *__restrict__ sums)
{
    __shared__ int warp_tot[kScanThreads / 32];
    const int ri = blockIdx.x;
    const Run &r = runs[ri];
    if (!r.state->do_sort) return;  // CTA-uniform
    const int b0 = seg.start[ri], nb = seg.start[ri + 1] - b0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int q0 = 0; q0 < nb; q0 += kScanThreads) {
        const int q = q0 + threadIdx.x;
        const int v = q < nb ? sums[b0 + q] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) {
            before += w < wid ? warp_tot[w] : 0;
            all += warp_tot[w];
        }
        if (q < nb) sums[b0 + q] = carry + before + inc - v;
        carry += all;
        __syncthreads();  // (warp_tot is rewritten by the next slice)
    }
    if (threadIdx.x == 0) r.tile_off[r.ntiles] = carry;
}

// Pass 3: block b adds the exclusive prefix of its run's block totals; the
// counters become the scatter cursors and tile_off[t] = cursor of key (t, 0).
__global__ void __launch_bounds__(kScanThreads) sort_scan_add_kernel(const Run *__restrict__ runs, Seg seg,
                                                                     const int *__restrict__ sums)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    if (!r.state->do_sort) return;  // CTA-uniform
    const int b0 = seg.start[ri], b = blockIdx.x;
    const int prefix = sums[b];
    const long long nk = (long long)r.ntiles * r.nsub;
    const long long k0 = (long long)(b - b0) * kScanChunk;
    for (int q = threadIdx.x; q < kScanChunk; q += blockDim.x) {
        const long long k = k0 + q;
        if (k >= nk) break;
        const int c = r.tile_cnt[k] + prefix;
        r.tile_cnt[k] = c;
        if ((k & (r.nsub - 1)) == 0) r.tile_off[k / r.nsub] = c;
    }
}

// Scatter: each CTA ranks its chunk's particles per key in shared memory
// (key table, warp match, shared atomics), reserves one contiguous range per
// key in the destination with one global atomic on its cursor, and copies
// every live particle to range start + rank.  Loads are 16-byte vector loads
// of four consecutive slots per thread (128 registers, two CTAs per SM: the
// kernel is bound by memory latency, and this keeps more bytes in flight than
// scalar loads at three CTAs per SM); for item j the lanes of a warp holding
// one key have consecutive ranks, so each store instruction writes a run of
// consecutive destination slots per key.
__global__ void __launch_bounds__(kSortThreads, 2) sort_scatter_kernel(const Run *__restrict__ runs, Seg seg,
                                                                    int32_t *__restrict__ src_out)
{
    __shared__ KeyTable t;
    for (int b = blockIdx.x; b < seg.nblocks; b += gridDim.x) {  // (CTA-uniform control flow)
        const int ri = seg_run(seg, b);
        const Run &r = runs[ri];
        if (!r.state->do_sort) {  // the run does not sort this step: skip its chunks
            b = next_own_chunk(seg.start[ri + 1]) - (int)gridDim.x;
            continue;
        }
        const KeyCtx kc = key_ctx(r, *r.state);
        const long long i0 = (long long)(b - seg.start[ri]) * kSortChunk;
        if (i0 >= kc.n_total) continue;
        const int buf = r.state->buf;
        const ParticleBuf src = r.P[buf];
        const ParticleBuf dst = r.P[buf ^ 1];
        int32_t cell[kSortItems];
#pragma unroll
        for (int g = 0; g < kSortItems / 4; ++g) load_cells4(src.cell, item_slot(i0, 4 * g), kc.n_total, cell + 4 * g);
        table_init(t);
        __syncthreads();
        const int lane = threadIdx.x & 31;
        const unsigned below = (1u << lane) - 1u;
        int slot[kSortItems], rank[kSortItems];
#pragma unroll
        for (int g = 0; g < kSortItems / 4; ++g) {
            int key[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                key[q] = sub_key(kc, key_of_cell(kc, cell[4 * g + q]), item_slot(i0, 4 * g + q), cell[4 * g + q]);
            if (__all_sync(0xffffffffu, key[0] == key[1] && key[0] == key[2] && key[0] == key[3])) {
                // each thread's four slots share a key: one item of weight 4
                // per thread; slot q of each peer lane gets rank q (peers) +
                // (peers below), so that one store instruction of the copy
                // writes consecutive addresses
                const unsigned peers = key_peers(key[0]);
                const int leader = __ffs(peers) - 1;
                int e = -2, off = 0;
                if (key[0] >= 0 && lane == leader) {
                    e = table_slot(t, key[0]);
                    off = e >= 0 ? atomicAdd(&t.cnt[e], 4 * __popc(peers))
                                 : atomicAdd(&r.tile_cnt[key[0]], 4 * __popc(peers));
                }
                e = __shfl_sync(0xffffffffu, e, leader);
                off = __shfl_sync(0xffffffffu, off, leader);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    slot[4 * g + q] = key[0] >= 0 ? e : -2;
                    rank[4 * g + q] = off + q * __popc(peers) + __popc(peers & below);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int key1 = key[q];
                    const unsigned peers = key_peers(key1);
                    const int leader = __ffs(peers) - 1;
                    int e = -2, off = 0;
                    if (key1 >= 0 && lane == leader) {
                        e = table_slot(t, key1);
                        off = e >= 0 ? atomicAdd(&t.cnt[e], __popc(peers)) : atomicAdd(&r.tile_cnt[key1], __popc(peers));
                    }
                    e = __shfl_sync(0xffffffffu, e, leader);
                    off = __shfl_sync(0xffffffffu, off, leader);
                    slot[4 * g + q] = key1 >= 0 ? e : -2;  // -2: dead or outside the window, -1: rank is absolute
                    rank[4 * g + q] = off + __popc(peers & below);
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kSortHash; e += blockDim.x)
            if (t.key[e] >= 0 && t.cnt[e] > 0) t.base[e] = atomicAdd(&r.tile_cnt[t.key[e]], t.cnt[e]);
        __syncthreads();
        const bool d3 = kc.dim == 3;
#pragma unroll
        for (int g = 0; g < kSortItems / 4; ++g) {
            const long long s0 = item_slot(i0, 4 * g);
            float o[3][4], u[3][4], wv[4];
            int32_t idv[4] = {0, 0, 0, 0};
            load4<float, float4>(src.off[0], s0, kc.n_total, o[0]);
            load4<float, float4>(src.off[1], s0, kc.n_total, o[1]);
            if (d3) load4<float, float4>(src.off[2], s0, kc.n_total, o[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) load4<float, float4>(src.u[a], s0, kc.n_total, u[a]);
            if (src.w) load4<float, float4>(src.w, s0, kc.n_total, wv);
            if (src.id) load4<int32_t, int4>(src.id, s0, kc.n_total, idv);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * g + q;
                if (slot[j] == -2) continue;
                const long long d = slot[j] >= 0 ? (long long)t.base[slot[j]] + rank[j] : (long long)rank[j];
                dst.cell[d] = cell[j];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (a < 2 || d3) dst.off[a][d] = o[a][q];
                    dst.u[a][d] = u[a][q];
                }
                if (src.w) dst.w[d] = wv[q];
                if (src.id) dst.id[d] = idv[q];
                if (src_out) src_out[d] = (int32_t)(s0 + q);
            }
        }
        __syncthreads();  // (the next chunk re-initialises the table)
    }
}

__global__ void sort_finish_kernel(const Run *__restrict__ runs, int nruns)
{
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    RunState &s = *r.state;
    if (!s.do_sort) return;
    s.buf ^= 1;
    s.n_sorted = r.tile_off[r.ntiles];
    s.n_total = s.n_sorted;
}

}  // namespace

cudaError_t launch_sort(const Run *runs, int nruns, Seg parts, Seg keys, int *scan_sums, int32_t *src_out,
                        int force, int max_interval, int adaptive, cudaStream_t st)
{
    sort_decide_kernel<<<(nruns + 127) / 128, 128, 0, st>>>(runs, nruns, force, max_interval, adaptive);
    sort_zero_kernel<<<dim3(1024, nruns), kBlock, 0, st>>>(runs, nruns);
    // count and scatter: a grid of a few CTAs per SM walks the chunks (a
    // run that does not sort costs each CTA one check, not one CTA per chunk)
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int g_count = parts.nblocks < 16 * sms ? parts.nblocks : 16 * sms;
    const int g_scatter = parts.nblocks < 8 * sms ? parts.nblocks : 8 * sms;
    sort_count_kernel<<<g_count > 0 ? g_count : 1, kSortThreads, 0, st>>>(runs, parts);
    sort_scan_local_kernel<<<keys.nblocks, kScanThreads, 0, st>>>(runs, keys, scan_sums);
    sort_scan_sums_kernel<<<nruns, kScanThreads, 0, st>>>(runs, keys, scan_sums);
    sort_scan_add_kernel<<<keys.nblocks, kScanThreads, 0, st>>>(runs, keys, scan_sums);
    sort_scatter_kernel<<<g_scatter > 0 ? g_scatter : 1, kSortThreads, 0, st>>>(runs, parts, src_out);
    sort_finish_kernel<<<(nruns + 127) / 128, 128, 0, st>>>(runs, nruns);
    return cudaGetLastError();
}

}  // namespace pic
