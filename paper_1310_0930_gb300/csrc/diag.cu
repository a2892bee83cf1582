// diag.cu -- particle load / readback and diagnostics of one run: charge
// density, energies, Gauss-law residual and the tile load imbalance
// (max / mean particles per occupied tile, the paper's imbalance metric of
// Sec. 3 taken over tiles instead of nodes).
#include "common.cuh"
#include "internal.h"

namespace pic {

namespace {

__global__ void pack_kernel(const Run *__restrict__ run, long long base, long long n, int dim,
                            const int32_t *__restrict__ cell, const float *__restrict__ off,
                            const float *__restrict__ u, const float *__restrict__ w)
{
    const Run &r = *run;
    RunState &s = *r.state;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ParticleBuf pb = r.P[s.buf];
    const long long o = base + i;
    int c[3] = {0, 0, 0};
    bool ok = true;
    for (int a = 0; a < dim; ++a) {
        c[a] = cell[(long long)a * n + i];
        float f = off[(long long)a * n + i];
        ok = ok && c[a] >= 0 && c[a] < r.n[a] && f >= 0.f && f < 1.f;
        pb.off[a][o] = f;
    }
    if (ok && r.open_last) {
        // the caller gives window-frame indices; storage is the ring
        int st = c[dim - 1] + s.origin;
        c[dim - 1] = st >= r.n[dim - 1] ? st - r.n[dim - 1] : st;
    }
    if (!ok) atomicOr(&s.status, kStatusBadIndex);
    pb.cell[o] = ok ? pack_cell(r, c[0], c[1], dim == 3 ? c[2] : 0) : -1;
    const float u0 = u[i], u1 = u[n + i], u2 = u[2 * n + i];
    pb.u[0][o] = u0;
    pb.u[1][o] = u1;
    pb.u[2][o] = u2;
    // a moving particle deposits current at the first step: its tile is
    // staged then, not streamed as a field-free tile (several threads may
    // store the same 1)
    if (ok && (u0 != 0.f || u1 != 0.f || u2 != 0.f) && r.fz) r.fz[tile_of(r, c[0], c[1], dim == 3 ? c[2] : 0)] = 1;
    if (pb.w) pb.w[o] = w ? w[i] : r.w_const;
    if (pb.id) pb.id[o] = (int32_t)o;
}

__global__ void set_count_kernel(const Run *__restrict__ run, long long n_total, int sorted)
{
    RunState &s = *run->state;
    s.n_total = n_total;
    if (sorted) s.n_sorted = n_total;
}

__device__ __forceinline__ bool live(const Run &r, const RunState &s, int32_t c, int &cx, int &cy, int &cz)
{
    if (c < 0) return false;
    unpack_cell(r, c, cx, cy, cz);
    if (r.open_last) {
        int pl = phys_last(r, s, r.dim == 3 ? cz : cy);
        if (pl < r.margin || pl >= r.n[r.dim - 1] - r.margin) return false;
    }
    return true;
}

// Charge density rho = sum_p q w S(x - x_i) at the nodes (Sec. 2), FP64
// sums.  Each CTA takes a chunk of kChargeChunk consecutive slots.  Slots
// are in tile order after a sort and in load order before (neighbouring
// slots hold neighbouring particles in both), so a chunk's node windows
// usually fit a small box: the CTA accumulates the chunk's values in that
// box in shared memory, as a fixed-point split of each value x = v S (the
// nearest integer of x and 12 bits of the remainder, two int32 words, with
// S = min(2^30 / sum |q w|, kChargeMax / max |q w|) over the chunk, so that
// no word overflows and each split is exact), and adds each non-zero box
// node to rho with one FP64 atomic.  The split represents each value to
// 2^-13 / S, below the FP32 rounding of the value itself.  A chunk whose box
// would exceed kChargeBox nodes (particles far apart: across a periodic
// seam, or a run in no particular order) adds every value to rho directly.
constexpr int kChargeChunk = 4096, kChargeItems = kChargeChunk / kBlock;
constexpr int kChargeBox = 5120;           // nodes of the shared box (two words each)
constexpr float kChargeRound = 12582912.f;  // 1.5 * 2^23: x + kChargeRound = 2^23 + 2^22 + rint(x), |x| < 2^22
constexpr int kChargeRoundBits = 0x4B400000;
constexpr float kChargeMax = 4.0e6f;  // bound on one scaled value (< 2^22)

template <int DIM, int P>
__global__ void __launch_bounds__(kBlock) charge_kernel(const Run *__restrict__ run, double *__restrict__ rho,
                                                        long long cap)
{
    __shared__ int box[2 * kChargeBox];
    __shared__ int s_lo[3], s_hi[3];
    __shared__ float s_sum;
    __shared__ unsigned s_max;
    const Run &r = *run;
    const RunState &s = *r.state;
    const long long i0 = (long long)blockIdx.x * kChargeChunk;
    if (i0 >= s.n_total) return;
    const ParticleBuf pb = r.P[s.buf];
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = 0x7fffffff;
        s_hi[threadIdx.x] = -0x7fffffff;
    }
    if (threadIdx.x == 0) {
        s_sum = 0.f;
        s_max = 0u;
    }
    __syncthreads();
    // the bounding box of the chunk's live cells and the scale bounds
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    float sum = 0.f, mx = 0.f;
#pragma unroll
    for (int k = 0; k < kChargeItems; ++k) {
        const long long i = i0 + (long long)k * kBlock + threadIdx.x;
        int c[3] = {0, 0, 0};
        if (i < s.n_total && live(r, s, pb.cell[i], c[0], c[1], c[2])) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                lo[a] = min(lo[a], c[a]);
                hi[a] = max(hi[a], c[a]);
            }
            const float aq = fabsf(r.q * (pb.w ? pb.w[i] : r.w_const));
            sum += aq;
            mx = fmaxf(mx, aq);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            atomicMin(&s_lo[a], lo[a]);
            atomicMax(&s_hi[a], hi[a]);
        }
        atomicAdd(&s_sum, sum);
        atomicMax(&s_max, __float_as_uint(mx));  // (non-negative floats order as their bits)
    }
    __syncthreads();
    if (s_hi[0] < s_lo[0]) return;  // (no live particle in the chunk; the same in every thread)
    constexpr int NL = P / 2;       // nodes below a particle's cell (nodes above: NL + 1)
    int org[3] = {0, 0, 0}, bd[3] = {1, 1, 1};
    long long nodes = 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        org[a] = s_lo[a] - NL;
        bd[a] = s_hi[a] - s_lo[a] + 2 * NL + 2;
        nodes *= bd[a];
    }
    const bool use_box = nodes <= kChargeBox;  // (the same in every thread)
    const float M = __uint_as_float(s_max), B = 1.01f * s_sum;
    if (!(M > 0.f)) return;  // (no charge in the chunk)
    const float S = fminf(1073741824.f / B, kChargeMax / M);
    if (use_box) {
        for (int q = threadIdx.x; q < 2 * (int)nodes; q += blockDim.x) box[q < (int)nodes ? q : kChargeBox + q - (int)nodes] = 0;
        __syncthreads();
    }
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1;
#pragma unroll 1
    for (int k = 0; k < kChargeItems; ++k) {
        const long long i = i0 + (long long)k * kBlock + threadIdx.x;
        int c[3] = {0, 0, 0};
        if (i >= s.n_total || !live(r, s, pb.cell[i], c[0], c[1], c[2])) continue;
        int base[3] = {0, 0, 0};
        float w[3][P + 1] = {};
#pragma unroll
        for (int a = 0; a < DIM; ++a) Shape<P>::node(c[a], pb.off[a][i], base[a], w[a]);
        const float qw = r.q * (pb.w ? pb.w[i] : r.w_const);
        if (use_box) {
            const float qs = qw * S;
            const int b0 = (base[0] - org[0]) + bd[0] * ((base[1] - org[1]) + bd[1] * (base[2] - org[2]));
#pragma unroll
            for (int qz = 0; qz < (DIM == 3 ? P + 1 : 1); ++qz)
#pragma unroll
                for (int qy = 0; qy <= P; ++qy)
#pragma unroll
                    for (int qx = 0; qx <= P; ++qx) {
                        const float x = qs * w[0][qx] * w[1][qy] * (DIM == 3 ? w[2][qz] : 1.f);
                        const float t = x + kChargeRound;          // kChargeRound + rint(x), exact
                        const float rem = x - (t - kChargeRound);  // x - rint(x), exact, |rem| <= 1/2
                        const float tl = fmaf(rem, 4096.f, kChargeRound);
                        const int q = b0 + qx + bd[0] * (qy + bd[1] * qz);
                        atomicAdd(&box[q], __float_as_int(t) - kChargeRoundBits);
                        atomicAdd(&box[kChargeBox + q], __float_as_int(tl) - kChargeRoundBits);
                    }
        } else {
            // node values in FP32 (one rounding per value), sums in FP64
#pragma unroll
            for (int qz = 0; qz < (DIM == 3 ? P + 1 : 1); ++qz)
#pragma unroll
                for (int qy = 0; qy <= P; ++qy)
#pragma unroll
                    for (int qx = 0; qx <= P; ++qx) {
                        const double v = (double)(qw * w[0][qx] * w[1][qy] * (DIM == 3 ? w[2][qz] : 1.f));
                        const int x = wrapi(base[0] + qx, n0), y = wrapi(base[1] + qy, n1);
                        const int z = DIM == 3 ? wrapi(base[2] + qz, n2) : 0;
                        atomicAdd(rho + x + (long long)n0 * (y + (long long)n1 * z), v);
                    }
        }
    }
    if (!use_box) return;
    __syncthreads();
    const double inv = 1.0 / (double)S, inv_lo = inv / 4096.0;
    for (int q = threadIdx.x; q < (int)nodes; q += blockDim.x) {
        const int vh = box[q], vl = box[kChargeBox + q];
        if ((vh | vl) == 0) continue;
        const int bx = q % bd[0], byz = q / bd[0], by = byz % bd[1], bz = byz / bd[1];
        const int x = modi(org[0] + bx, n0), y = modi(org[1] + by, n1), z = DIM == 3 ? modi(org[2] + bz, n2) : 0;
        atomicAdd(rho + x + (long long)n0 * (y + (long long)n1 * z), (double)vh * inv + (double)vl * inv_lo);
    }
    (void)cap;
}

__device__ __forceinline__ unsigned long long warp_slot(unsigned long long *count, bool want)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, want);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader && m) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(act, base, leader);
    return base + __popc(m & ((1u << lane) - 1));
}

__global__ void unpack_kernel(const Run *__restrict__ run, long long cap, int dim, int32_t *cell, float *off,
                              float *u, float *w, int32_t *id, unsigned long long *count)
{
    const Run &r = *run;
    const RunState &s = *r.state;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const ParticleBuf pb = r.P[s.buf];
    int c[3] = {0, 0, 0};
    const bool ok = i < s.n_total && live(r, s, pb.cell[i], c[0], c[1], c[2]);
    const unsigned long long o = warp_slot(count, ok);
    if (!ok || (long long)o >= cap) return;
    if (r.open_last) c[dim - 1] = phys_last(r, s, c[dim - 1]);
    for (int a = 0; a < dim; ++a) {
        if (cell) cell[(long long)a * cap + o] = c[a];
        if (off) off[(long long)a * cap + o] = pb.off[a][i];
    }
    if (u) {
        u[o] = pb.u[0][i];
        u[cap + o] = pb.u[1][i];
        u[2 * cap + o] = pb.u[2][i];
    }
    if (w) w[o] = pb.w ? pb.w[i] : r.w_const;
    if (id) id[o] = pb.id ? pb.id[i] : -1;
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void field_energy_kernel(const Run *__restrict__ run, double *out)
{
    const Run &r = *run;
    __shared__ double sh[32];
    double e2 = 0.0, b2 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.ncell; i += gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            double e = r.E[c][i], b = r.B[c][i];
            e2 += e * e;
            b2 += b * b;
        }
    double te = block_sum(e2, sh);
    double tb = block_sum(b2, sh);
    if (threadIdx.x == 0) {
        atomicAdd(out + 0, te);
        atomicAdd(out + 1, tb);
    }
}

__global__ void kinetic_kernel(const Run *__restrict__ run, double *out)
{
    const Run &r = *run;
    const RunState &s = *r.state;
    __shared__ double sh[32];
    const ParticleBuf pb = r.P[s.buf];
    double k = 0.0, cnt = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < s.n_total;
         i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        if (!live(r, s, pb.cell[i], c[0], c[1], c[2])) continue;
        // gamma - 1 = u^2 / (gamma + 1): no cancellation in FP32; sums in FP64
        const float ux = pb.u[0][i], uy = pb.u[1][i], uz = pb.u[2][i];
        const float u2 = ux * ux + uy * uy + uz * uz;
        const float gm1 = u2 / (sqrtf(1.f + u2) + 1.f);
        k += (double)((pb.w ? pb.w[i] : r.w_const) * r.m * gm1);
        cnt += 1.0;
    }
    double tk = block_sum(k, sh);
    double tc = block_sum(cnt, sh);
    if (threadIdx.x == 0) {
        atomicAdd(out + 2, tk);
        atomicAdd(out + 3, tc);
    }
}

template <int DIM>
__global__ void gauss_kernel(const Run *__restrict__ run, const double *__restrict__ rho, unsigned *umax)
{
    const Run &r = *run;
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1;
    const double id0 = 1.0 / r.dd[0], id1 = 1.0 / r.dd[1], id2 = DIM == 3 ? 1.0 / r.dd[2] : 0.0;
    float mr = 0.f, m0 = 0.f;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < r.ncell; idx += gridDim.x * blockDim.x) {
        int i = idx % n0, j = (idx / n0) % n1, k = DIM == 3 ? idx / (n0 * n1) : 0;
        int mx = (i == 0 ? n0 - 1 : i - 1) + n0 * (j + n1 * k);
        int my = i + n0 * ((j == 0 ? n1 - 1 : j - 1) + n1 * k);
        double dv = ((double)r.E[0][idx] - r.E[0][mx]) * id0 + ((double)r.E[1][idx] - r.E[1][my]) * id1;
        if (DIM == 3) {
            int mz = i + n0 * (j + n1 * (k == 0 ? n2 - 1 : k - 1));
            dv += ((double)r.E[2][idx] - r.E[2][mz]) * id2;
        }
        double res = dv - (rho[idx] - r.rho0[idx]);
        mr = fmaxf(mr, (float)fabs(res));
        m0 = fmaxf(m0, (float)fabs(r.rho0[idx]));
    }
    atomicMax(umax + 0, __float_as_uint(mr));
    atomicMax(umax + 1, __float_as_uint(m0));
}

__global__ void tiles_kernel(const Run *__restrict__ run, unsigned *umax)
{
    const Run &r = *run;
    unsigned mx = 0, occ = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r.ntiles; t += gridDim.x * blockDim.x) {
        unsigned c = (unsigned)(r.tile_off[t + 1] - r.tile_off[t]);
        mx = c > mx ? c : mx;
        occ += c > 0;
    }
    atomicMax(umax + 2, mx);
    atomicAdd(umax + 3, occ);
}

}  // namespace

cudaError_t launch_pack(const Run *run, long long base, long long n, int dim, const int32_t *cell,
                        const float *off, const float *u, const float *w, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    pack_kernel<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(run, base, n, dim, cell, off, u, w);
    return cudaGetLastError();
}

cudaError_t launch_set_count(const Run *run, long long n_total, int sorted, cudaStream_t st)
{
    set_count_kernel<<<1, 1, 0, st>>>(run, n_total, sorted);
    return cudaGetLastError();
}

__global__ void to_float_kernel(const double *__restrict__ src, float *__restrict__ dst, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

cudaError_t launch_to_float(const double *src, float *dst, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    to_float_kernel<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_charge(int dim, int order, const Run *run, double *rho, long long cap, cudaStream_t st)
{
    unsigned g = (unsigned)((cap + kChargeChunk - 1) / kChargeChunk);
    if (g == 0) return cudaSuccess;
    if (dim == 2) {
        if (order == 1) charge_kernel<2, 1><<<g, kBlock, 0, st>>>(run, rho, cap);
        else if (order == 2) charge_kernel<2, 2><<<g, kBlock, 0, st>>>(run, rho, cap);
        else if (order == 3) charge_kernel<2, 3><<<g, kBlock, 0, st>>>(run, rho, cap);
        else charge_kernel<2, 4><<<g, kBlock, 0, st>>>(run, rho, cap);
    } else {
        if (order == 1) charge_kernel<3, 1><<<g, kBlock, 0, st>>>(run, rho, cap);
        else if (order == 2) charge_kernel<3, 2><<<g, kBlock, 0, st>>>(run, rho, cap);
        else if (order == 3) charge_kernel<3, 3><<<g, kBlock, 0, st>>>(run, rho, cap);
        else charge_kernel<3, 4><<<g, kBlock, 0, st>>>(run, rho, cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Run *run, long long cap, int dim, int32_t *cell, float *off, float *u, float *w,
                          int32_t *id, unsigned long long *count, cudaStream_t st)
{
    unsigned g = (unsigned)((cap + kBlock - 1) / kBlock);
    if (g == 0) return cudaSuccess;
    unpack_kernel<<<g, kBlock, 0, st>>>(run, cap, dim, cell, off, u, w, id, count);
    return cudaGetLastError();
}

cudaError_t launch_diag(int dim, const Run *run, const double *rho, long long cap, double *out, cudaStream_t st)
{
    unsigned *umax = reinterpret_cast<unsigned *>(out + 8);
    field_energy_kernel<<<1024, kBlock, 0, st>>>(run, out);
    kinetic_kernel<<<1024, kBlock, 0, st>>>(run, out);
    if (dim == 3) gauss_kernel<3><<<1024, kBlock, 0, st>>>(run, rho, umax);
    else gauss_kernel<2><<<1024, kBlock, 0, st>>>(run, rho, umax);
    tiles_kernel<<<256, kBlock, 0, st>>>(run, umax);
    (void)cap;
    return cudaGetLastError();
}

}  // namespace pic
