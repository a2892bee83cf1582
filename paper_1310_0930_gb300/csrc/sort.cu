// sort.cu -- periodic counting sort of the particles by tile.
//
// The GPU counterpart of the paper's particle migration between nodes after
// the push (Sec. 3): particles that moved are regrouped with the tile that
// now owns them, dead slots (absorbed particles) are dropped, and the tail
// of freshly injected plasma is merged.  Steps, per run:
//   1. zero the tile counters;
//   2. histogram of tile keys (warp-aggregated atomics: neighbouring
//      particles mostly share a tile);
//   3. exclusive scan of the counts into tile offsets (one CTA per run);
//   4. scatter every live particle into the alternate buffer at
//      offset[key] + rank (rank from warp-aggregated cursor atomics);
//   5. flip the buffer and set the sorted count.
// Order within a tile is not stable (cursor atomics); nothing downstream
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

// tile key of slot i, or -1 for a dead slot / a particle outside the window
__device__ __forceinline__ int key_of(const Run &r, const RunState &s, const ParticleBuf &pb, long long i)
{
    if (i >= s.n_total) return -1;
    int32_t c = pb.cell[i];
    if (c < 0) return -1;
    int cx, cy, cz;
    unpack_cell(r, c, cx, cy, cz);
    if (r.open_last) {
        int pl = phys_last(r, s, r.dim == 3 ? cz : cy);
        if (pl < r.margin || pl >= r.n[r.dim - 1] - r.margin) return -1;
    }
    return tile_of(r, cx, cy, cz);
}

__global__ void sort_zero_kernel(const Run *__restrict__ runs, int nruns, int max_tiles)
{
    const int ri = blockIdx.y;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r.ntiles; t += gridDim.x * blockDim.x)
        r.tile_cnt[t] = 0;
}

__global__ void sort_count_kernel(const Run *__restrict__ runs, Seg seg)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    const RunState &s = *r.state;
    const long long i = (long long)(blockIdx.x - seg.start[ri]) * blockDim.x + threadIdx.x;
    const ParticleBuf pb = r.P[s.buf];
    const int key = key_of(r, s, pb, i);
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&r.tile_cnt[key], __popc(peers));
}

// One CTA per run: tile_off = exclusive scan of tile_cnt; tile_cnt becomes
// the scatter cursor (= tile_off).
__global__ void __launch_bounds__(1024) sort_scan_kernel(const Run *__restrict__ runs, int nruns)
{
    const int ri = blockIdx.x;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    const int nt = r.ntiles;
    const int per = (nt + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per;
    const int hi = lo + per < nt ? lo + per : nt;
    long long sum = 0;
    for (int t = lo; t < hi; ++t) sum += r.tile_cnt[t];
    __shared__ long long part[1024];
    part[threadIdx.x] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan over the per-thread partial sums
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        long long v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;
    for (int t = lo; t < hi; ++t) {
        int c = r.tile_cnt[t];
        r.tile_off[t] = (int32_t)run;
        r.tile_cnt[t] = (int32_t)run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) r.tile_off[nt] = (int32_t)part[blockDim.x - 1];
}

__global__ void sort_scatter_kernel(const Run *__restrict__ runs, Seg seg)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    const RunState &s = *r.state;
    const long long i = (long long)(blockIdx.x - seg.start[ri]) * blockDim.x + threadIdx.x;
    const ParticleBuf src = r.P[s.buf];
    const ParticleBuf dst = r.P[s.buf ^ 1];
    const int key = key_of(r, s, src, i);
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (key >= 0 && lane == leader) base = atomicAdd(&r.tile_cnt[key], __popc(peers));
    base = __shfl_sync(act, base, leader);
    if (key < 0) return;
    const long long o = base + __popc(peers & ((1u << lane) - 1));
    dst.cell[o] = src.cell[i];
    for (int a = 0; a < r.dim; ++a) dst.off[a][o] = src.off[a][i];
    dst.u[0][o] = src.u[0][i];
    dst.u[1][o] = src.u[1][i];
    dst.u[2][o] = src.u[2][i];
    if (src.w) dst.w[o] = src.w[i];
    if (src.id) dst.id[o] = src.id[i];
}

__global__ void sort_finish_kernel(const Run *__restrict__ runs, int nruns)
{
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    RunState &s = *r.state;
    s.buf ^= 1;
    s.n_sorted = r.tile_off[r.ntiles];
    s.n_total = s.n_sorted;
}

}  // namespace

cudaError_t launch_sort(const Run *runs, int nruns, Seg parts, int max_tiles, cudaStream_t st)
{
    dim3 zg((max_tiles + kBlock - 1) / kBlock < 4096 ? (max_tiles + kBlock - 1) / kBlock : 4096, nruns);
    sort_zero_kernel<<<zg, kBlock, 0, st>>>(runs, nruns, max_tiles);
    sort_count_kernel<<<parts.nblocks, kBlock, 0, st>>>(runs, parts);
    sort_scan_kernel<<<nruns, 1024, 0, st>>>(runs, nruns);
    sort_scatter_kernel<<<parts.nblocks, kBlock, 0, st>>>(runs, parts);
    sort_finish_kernel<<<(nruns + 127) / 128, 128, 0, st>>>(runs, nruns);
    return cudaGetLastError();
}

}  // namespace pic
