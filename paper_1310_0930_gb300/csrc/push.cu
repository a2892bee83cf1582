// push.cu -- dispatch of the particle kernel over the compiled tile menu, the
// per-step classification of tiles into live and zero-field ones, and the
// zero-field streaming kernel.
#include "push.cuh"

namespace pic {

cudaError_t launch_push_2d(int, const int *, int, const PushArgs &, cudaStream_t);
cudaError_t launch_push_3d_a(int, const int *, int, const PushArgs &, cudaStream_t);
cudaError_t launch_push_3d_b(int, const int *, int, const PushArgs &, cudaStream_t);
cudaError_t launch_push_3d_tma(int, const int *, int, const PushArgs &, cudaStream_t);
size_t smem_push_2d(int, const int *, int);
size_t smem_push_3d_a(int, const int *, int);
size_t smem_push_3d_b(int, const int *, int);
size_t smem_push_3d_tma(int, const int *, int);
int stage_push_2d(int, const int *, int, int *, int *);
int stage_push_3d_a(int, const int *, int, int *, int *);
int stage_push_3d_b(int, const int *, int, int *, int *);
int stage_push_3d_tma(int, const int *, int, int *, int *);
int box_push_3d_tma(int, const int *, int, int *);
cudaError_t launch_push_q(int, const int *, int, const PushArgs &, cudaStream_t);
size_t smem_push_q(int, const int *, int);
int stage_push_q(int, const int *, int, int *, int *);
cudaError_t launch_push_split(int, int, const int *, int, const PushArgs &, cudaStream_t);
size_t smem_push_split(int, int, const int *, int);
int stage_push_split(int, int, const int *, int, int *, int *);

int push_default_drift(int dim, const int *tile)
{
    if (dim == 3) return 1;
    if (tile[0] == 16) return 2;
    if (tile[0] == 8) return 1;
    return 2;
}

size_t push_smem_bytes(int dim, int order, const int *tile, int drift, int variant)
{
    if (variant == 2) return smem_push_split(dim, order, tile, drift);
    const bool tma = variant == 1;
    if (order == 4) return tma ? 0 : smem_push_q(dim, tile, drift);
    if (dim == 2) return tma ? 0 : smem_push_2d(order, tile, drift);
    if (tma) return smem_push_3d_tma(order, tile, drift);
    size_t s = smem_push_3d_a(order, tile, drift);
    return s ? s : smem_push_3d_b(order, tile, drift);
}

int push_tma_box(int dim, int order, const int *tile, int drift, int *box)
{
    return dim == 3 && order <= 3 ? box_push_3d_tma(order, tile, drift, box) : 0;
}

int push_stage_extent(int dim, int order, const int *tile, int drift, int variant, int *lo, int *len)
{
    if (variant == 2) return stage_push_split(dim, order, tile, drift, lo, len);
    const bool tma = variant == 1;
    if (order == 4) return tma ? 0 : stage_push_q(dim, tile, drift, lo, len);
    if (dim == 2) return tma ? 0 : stage_push_2d(order, tile, drift, lo, len);
    if (tma) return stage_push_3d_tma(order, tile, drift, lo, len);
    return stage_push_3d_a(order, tile, drift, lo, len) || stage_push_3d_b(order, tile, drift, lo, len);
}

cudaError_t launch_push(int dim, int order, const int *tile, int drift, int variant, const PushArgs &a,
                        cudaStream_t st)
{
    if (variant == 2) return launch_push_split(dim, order, tile, drift, a, st);
    const bool tma = variant == 1;
    if (order == 4) return tma ? cudaErrorInvalidValue : launch_push_q(dim, tile, drift, a, st);
    if (dim == 2) return launch_push_2d(order, tile, drift, a, st);
    if (tma) return launch_push_3d_tma(order, tile, drift, a, st);
    if (smem_push_3d_a(order, tile, drift)) return launch_push_3d_a(order, tile, drift, a, st);
    return launch_push_3d_b(order, tile, drift, a, st);
}

namespace {

constexpr int kMaxBricks = 8;  // tiles one axis of a staged region may touch (else: taken as live)

// Tiles (along one axis of n cells, tiles of 2^tlog cells) that hold the cells
// [lo, lo + len) wrapped periodically; returns their count, or kMaxBricks + 1.
__device__ int tiles_on_axis(int lo, int len, int n, int tlog, int *out)
{
    int cnt = 0;
    while (len > 0) {
        if (cnt == kMaxBricks) return kMaxBricks + 1;
        const int c = modi(lo, n);
        const int t = c >> tlog;
        int end = (t + 1) << tlog;
        end = end < n ? end : n;
        const int step = end - c < len ? end - c : len;
        bool seen = false;
        for (int q = 0; q < cnt; ++q) seen = seen || out[q] == t;
        if (!seen) out[cnt++] = t;
        lo += step;
        len -= step;
    }
    return cnt;
}

}  // namespace

__global__ void classify_tiles_kernel(const Run *__restrict__ runs, const Item *__restrict__ items, int n_tail,
                                      int n_items, int3 stage_lo, int3 stage_len, Item *__restrict__ live,
                                      Item *__restrict__ zero, int *__restrict__ cnt)
{
    const int i = n_tail + blockIdx.x * blockDim.x + threadIdx.x;
    Item it{0, 0, 0, 0};
    bool take = false, is_live = true;
    if (i < n_items) {
        it = items[i];
        const Run &r = runs[it.run];
        const int t = it.a;
        take = r.tile_off[t + 1] > r.tile_off[t];
        if (take && r.fz) {
            const int tc[3] = {t % r.nt[0], (t / r.nt[0]) % r.nt[1], t / (r.nt[0] * r.nt[1])};
            const int lo[3] = {stage_lo.x, stage_lo.y, stage_lo.z}, len[3] = {stage_len.x, stage_len.y, stage_len.z};
            int tl[3][kMaxBricks], nb[3] = {1, 1, 1};
            tl[1][0] = tl[2][0] = 0;
            bool ok = true;
            for (int a = 0; a < r.dim; ++a) {
                nb[a] = tiles_on_axis((tc[a] << r.tlog[a]) - lo[a], len[a], r.n[a], r.tlog[a], tl[a]);
                ok = ok && nb[a] <= kMaxBricks;
            }
            if (ok) {
                unsigned any = 0;
                for (int z = 0; z < nb[2]; ++z)
                    for (int y = 0; y < nb[1]; ++y)
                        for (int x = 0; x < nb[0]; ++x)
                            any |= r.fz[tl[0][x] + r.nt[0] * (tl[1][y] + r.nt[1] * tl[2][z])];
                is_live = any != 0;
            }
        }
    }
    // warp-aggregated appends (items of one warp keep their order)
    const unsigned lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
    const unsigned m_live = __ballot_sync(0xffffffffu, take && is_live);
    {  // live tiles per run (diagnostics): one atomic per run and warp
        const unsigned peers = __match_any_sync(0xffffffffu, take && is_live ? it.run : -1);
        if (take && is_live && lane == (unsigned)(__ffs(peers) - 1))
            atomicAdd(&runs[it.run].state->live_tiles, (unsigned long long)__popc(peers));
    }
    const unsigned m_zero = __ballot_sync(0xffffffffu, take && !is_live);
    int b_live = 0, b_zero = 0;
    if (lane == 0) {
        if (m_live) b_live = atomicAdd(cnt + 0, __popc(m_live));
        if (m_zero) b_zero = atomicAdd(cnt + 1, __popc(m_zero));
    }
    b_live = __shfl_sync(0xffffffffu, b_live, 0);
    b_zero = __shfl_sync(0xffffffffu, b_zero, 0);
    if (take && is_live) live[n_tail + b_live + __popc(m_live & lt)] = it;
    if (take && !is_live) zero[b_zero + __popc(m_zero & lt)] = it;
}

cudaError_t launch_classify(const Run *runs, const Item *items, int n_tail, int n_items, const int *stage_lo,
                            const int *stage_len, Item *live, Item *zero, int *cnt, cudaStream_t st)
{
    const int n = n_items - n_tail;
    if (n <= 0) return cudaSuccess;
    const int3 lo = make_int3(stage_lo[0], stage_lo[1], stage_lo[2]);
    const int3 len = make_int3(stage_len[0], stage_len[1], stage_len[2]);
    classify_tiles_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(runs, items, n_tail, n_items, lo, len, live,
                                                                        zero, cnt);
    return cudaGetLastError();
}

cudaError_t launch_push_zero(int dim, int order, bool split, const Run *runs, const Item *zero, const int *count,
                             int max_items, int num_sms, bool wide, cudaStream_t st)
{
    using namespace push_detail;
    if (split) {  // (moving particles of zero-field tiles deposit as virtual trajectories)
        if (dim == 2) {
            if (order == 1) return launch_zero<2, 1, true>(runs, zero, count, max_items, num_sms, wide, st);
            if (order == 2) return launch_zero<2, 2, true>(runs, zero, count, max_items, num_sms, wide, st);
            return launch_zero<2, 3, true>(runs, zero, count, max_items, num_sms, wide, st);
        }
        if (order == 1) return launch_zero<3, 1, true>(runs, zero, count, max_items, num_sms, wide, st);
        if (order == 2) return launch_zero<3, 2, true>(runs, zero, count, max_items, num_sms, wide, st);
        return launch_zero<3, 3, true>(runs, zero, count, max_items, num_sms, wide, st);
    }
    if (dim == 2) {
        if (order == 1) return launch_zero<2, 1>(runs, zero, count, max_items, num_sms, wide, st);
        if (order == 2) return launch_zero<2, 2>(runs, zero, count, max_items, num_sms, wide, st);
        if (order == 3) return launch_zero<2, 3>(runs, zero, count, max_items, num_sms, wide, st);
        return launch_zero<2, 4>(runs, zero, count, max_items, num_sms, wide, st);
    }
    if (order == 1) return launch_zero<3, 1>(runs, zero, count, max_items, num_sms, wide, st);
    if (order == 2) return launch_zero<3, 2>(runs, zero, count, max_items, num_sms, wide, st);
    if (order == 3) return launch_zero<3, 3>(runs, zero, count, max_items, num_sms, wide, st);
    return launch_zero<3, 4>(runs, zero, count, max_items, num_sms, wide, st);
}

}  // namespace pic
