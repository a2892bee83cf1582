// push.cu -- fused particle kernel of the EM-PIC timestep (Sec. 5.2 steps
// i-v): per particle, B-spline weights -> gather of E and B at the Yee
// locations -> relativistic Boris push -> move on (cell, offset) -> Esirkepov
// charge-conserving current deposit.
//
// One CTA per tile (a block of cells): the tile's E and B plus a halo are
// staged in shared memory, its particles (sorted by tile) are loaded
// coalesced from the structure-of-arrays buffers, the current of the whole
// tile is accumulated in a shared-memory J tile (the GPU form of the paper's
// per-thread current copies, Sec. 3.1) and flushed to global J once with
// atomics (the paper's reduction of the copies).  A particle that strayed
// further than `drift` cells out of its tile since the last sort, and every
// particle of the unsorted tail (freshly injected plasma), takes the slow
// path: the same arithmetic on global memory with global atomics.
#include "common.cuh"
#include "internal.h"

namespace pic {

namespace {

// Gather of component C: sum_{a,b,c} wx[a] wy[b] wz[c] F_C(bx+a, by+b, bz+c).
template <int DIM, int P, int C, class F>
__device__ __forceinline__ float gather1(const F &f, int bx, int by, int bz, const float *wx,
                                         const float *wy, const float *wz)
{
    float s = 0.f;
    if (DIM == 3) {
#pragma unroll
        for (int c = 0; c <= P; ++c) {
            float sy = 0.f;
#pragma unroll
            for (int b = 0; b <= P; ++b) {
                float sx = 0.f;
#pragma unroll
                for (int a = 0; a <= P; ++a) sx = fmaf(wx[a], f(C, bx + a, by + b, bz + c), sx);
                sy = fmaf(wy[b], sx, sy);
            }
            s = fmaf(wz[c], sy, s);
        }
    } else {
#pragma unroll
        for (int b = 0; b <= P; ++b) {
            float sx = 0.f;
#pragma unroll
            for (int a = 0; a <= P; ++a) sx = fmaf(wx[a], f(C, bx + a, by + b, 0), sx);
            s = fmaf(wy[b], sx, s);
        }
    }
    return s;
}

// The six staged components in tile-local shared memory: (i,j,k) relative to
// the tile origin, shifted by the halo; component c at f + c*vol.
struct SmemFields {
    const float *f;
    int vol, hx, hy, hz, sx, sxy;
    __device__ __forceinline__ float operator()(int c, int i, int j, int k) const
    {
        return f[c * vol + (i + hx) + sx * (j + hy) + sxy * (k + hz)];
    }
};

// The six components in global memory, absolute indices wrapped periodically.
struct GlobalFields {
    const float *p[6];
    int n0, n1, n2;
    __device__ __forceinline__ float operator()(int c, int i, int j, int k) const
    {
        i = wrapi(i, n0);
        j = wrapi(j, n1);
        k = n2 > 1 ? wrapi(k, n2) : 0;
        return __ldg(p[c] + i + n0 * (j + n1 * k));
    }
};

struct SmemAcc {
    float *J;  // [3][vol]
    int vol, hx, hy, hz, sx, sxy;
    __device__ __forceinline__ void operator()(int comp, int i, int j, int k, float v) const
    {
        if (v != 0.f) atomicAdd(J + comp * vol + (i + hx) + sx * (j + hy) + sxy * (k + hz), v);
    }
};

struct GlobalAcc {
    float *J0, *J1, *J2;
    int n0, n1, n2;
    __device__ __forceinline__ void operator()(int comp, int i, int j, int k, float v) const
    {
        if (v == 0.f) return;
        i = wrapi(i, n0);
        j = wrapi(j, n1);
        k = n2 > 1 ? wrapi(k, n2) : 0;
        float *J = comp == 0 ? J0 : (comp == 1 ? J1 : J2);
        atomicAdd(J + i + n0 * (j + n1 * k), v);
    }
};

// Place the P+1 shape values `s` into a P+2 window at offset o (0 or 1)
// with compile-time indexing only (no local-memory arrays).
template <int P>
__device__ __forceinline__ void place(const float *s, int o, float *dst)
{
#pragma unroll
    for (int q = 0; q < P + 2; ++q) {
        float lo = q <= P ? s[q] : 0.f;
        float hi = q >= 1 ? s[q - 1] : 0.f;
        dst[q] = o ? hi : lo;
    }
}

// Esirkepov deposit of one straight move (Sec. 5.2 charge-conserving
// deposit): per axis the old and new node shapes on a (P+2)-node window,
// DS = S1 - S0, A = S0 + DS/2; then
//   3D: J_a(window) = coef_a * prefix_a(DS_a) * (A_b A_c + DS_b DS_c / 12),
//   2D: J_x = coef_x prefix_x(DS_x) A_y, J_y = coef_y prefix_y(DS_y) A_x,
//       J_z = q w v_z (A_x A_y + DS_x DS_y / 12),
// coef_a = -q w d_a / dt.  (A_b A_c + DS_b DS_c/12 equals the textbook
// S0S0 + DS S0/2 + S0 DS/2 + DS DS/3.)
template <int DIM, int P, class Acc>
__device__ __forceinline__ void esirkepov(const Acc &acc, const int *c0, const float *d0, const int *k,
                                          const float *d1, const float *coef, float qwvz)
{
    constexpr int W = P + 2;
    float A[DIM][W], DS[DIM][W];
    int wb[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int bo, bn;
        float so[P + 1], sn[P + 1], S0[W], S1[W];
        Shape<P>::node(c0[a], d0[a], bo, so);
        Shape<P>::node(c0[a] + k[a], d1[a], bn, sn);
        int s = bn - bo;  // -1, 0 or +1 for a move of less than one cell
        wb[a] = s < 0 ? bn : bo;
        place<P>(so, s < 0 ? 1 : 0, S0);
        place<P>(sn, s > 0 ? 1 : 0, S1);
#pragma unroll
        for (int q = 0; q < W; ++q) {
            DS[a][q] = S1[q] - S0[q];
            A[a][q] = S0[q] + 0.5f * DS[a][q];
        }
    }
    const float twelfth = 1.f / 12.f;
    if (DIM == 3) {
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const int a = comp, b = (comp + 1) % 3, c = (comp + 2) % 3;
            float Pa[W - 1];
            float run = 0.f;
#pragma unroll
            for (int q = 0; q < W - 1; ++q) {
                run += DS[a][q];
                Pa[q] = coef[a] * run;
            }
#pragma unroll
            for (int qc = 0; qc < W; ++qc)
#pragma unroll
                for (int qb = 0; qb < W; ++qb) {
                    float fac = fmaf(DS[b][qb] * twelfth, DS[c][qc], A[b][qb] * A[c][qc]);
#pragma unroll
                    for (int qa = 0; qa < W - 1; ++qa) {
                        int idx[3];
                        idx[a] = wb[a] + qa;
                        idx[b] = wb[b] + qb;
                        idx[c] = wb[c] + qc;
                        acc(comp, idx[0], idx[1], idx[2], Pa[qa] * fac);
                    }
                }
        }
    } else {
        float Px[W - 1], Py[W - 1];
        float rx = 0.f, ry = 0.f;
#pragma unroll
        for (int q = 0; q < W - 1; ++q) {
            rx += DS[0][q];
            ry += DS[1][q];
            Px[q] = coef[0] * rx;
            Py[q] = coef[1] * ry;
        }
#pragma unroll
        for (int qb = 0; qb < W; ++qb)
#pragma unroll
            for (int qa = 0; qa < W; ++qa) {
                if (qa < W - 1) acc(0, wb[0] + qa, wb[1] + qb, 0, Px[qa] * A[1][qb]);
                if (qb < W - 1) acc(1, wb[0] + qa, wb[1] + qb, 0, Py[qb] * A[0][qa]);
                acc(2, wb[0] + qa, wb[1] + qb, 0,
                    qwvz * fmaf(DS[0][qa] * twelfth, DS[1][qb], A[0][qa] * A[1][qb]));
            }
    }
}

// Relativistic Boris push (Sec. 5.2 step iii): half electric kick, rotation
// with t = (q dt / 2 m gamma) B and s = 2t/(1+t^2), half electric kick.
__device__ __forceinline__ void boris(float h, const float *e, const float *b, float *u)
{
    float um0 = fmaf(h, e[0], u[0]), um1 = fmaf(h, e[1], u[1]), um2 = fmaf(h, e[2], u[2]);
    float ig = rsqrtf(1.f + um0 * um0 + um1 * um1 + um2 * um2);
    float t0 = h * b[0] * ig, t1 = h * b[1] * ig, t2 = h * b[2] * ig;
    float f = 2.f / (1.f + t0 * t0 + t1 * t1 + t2 * t2);
    float s0 = f * t0, s1 = f * t1, s2 = f * t2;
    float p0 = um0 + (um1 * t2 - um2 * t1);
    float p1 = um1 + (um2 * t0 - um0 * t2);
    float p2 = um2 + (um0 * t1 - um1 * t0);
    u[0] = fmaf(h, e[0], um0 + (p1 * s2 - p2 * s1));
    u[1] = fmaf(h, e[1], um1 + (p2 * s0 - p0 * s2));
    u[2] = fmaf(h, e[2], um2 + (p0 * s1 - p1 * s0));
}

// Yee locations: E0 (h,n,n) E1 (n,h,n) E2 (n,n,h) B0 (n,h,h) B1 (h,n,h)
// B2 (h,h,n), h = half-integer, n = integer; in 2D the third entry is unused.
template <int DIM, int P, class F>
__device__ __forceinline__ void gather_all(const F &f, const int *bn, const int *bh, const float (*wn)[P + 1],
                                           const float (*wh)[P + 1], float *e, float *b)
{
    const int z_n = DIM == 3 ? bn[DIM - 1] : 0, z_h = DIM == 3 ? bh[DIM - 1] : 0;
    const float *wzn = wn[DIM - 1], *wzh = wh[DIM - 1];
    e[0] = gather1<DIM, P, 0>(f, bh[0], bn[1], z_n, wh[0], wn[1], wzn);
    e[1] = gather1<DIM, P, 1>(f, bn[0], bh[1], z_n, wn[0], wh[1], wzn);
    e[2] = gather1<DIM, P, 2>(f, bn[0], bn[1], z_h, wn[0], wn[1], wzh);
    b[0] = gather1<DIM, P, 3>(f, bn[0], bh[1], z_h, wn[0], wh[1], wzh);
    b[1] = gather1<DIM, P, 4>(f, bh[0], bn[1], z_h, wh[0], wn[1], wzh);
    b[2] = gather1<DIM, P, 5>(f, bh[0], bh[1], z_n, wh[0], wh[1], wzn);
}

// One particle through the whole step.  cr: cell coordinates in the frame
// of the accessors (tile-relative for shared memory, absolute for global).
// Returns false (and deposits nothing) when the move is not a finite move of
// less than one cell per axis, which only corrupted input can produce.
template <int DIM, int P, class F, class Acc>
__device__ __forceinline__ bool advance(const Run &r, const F &f, const Acc &acc, const int *cr, float *d,
                                        float *u, float w, int *kout)
{
    int bn[DIM], bh[DIM];
    float wn[DIM][P + 1], wh[DIM][P + 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        Shape<P>::node(cr[a], d[a], bn[a], wn[a]);
        Shape<P>::half(cr[a], d[a], bh[a], wh[a]);
    }
    float e[3], b[3];
    gather_all<DIM, P>(f, bn, bh, wn, wh, e, b);
    boris(r.qm_half_dt, e, b, u);
    float ig = rsqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    float d1[DIM];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        float nd = d[a] + r.dt_over_d[a] * u[a] * ig;
        ok = ok && nd > -1.f && nd < 2.f;  // false for NaN too
        nd = ok ? nd : d[a];
        float k = floorf(nd);
        nd = nd - k;
        if (nd >= 1.f) {  // FP32 rounding of a value just below an integer
            nd = 0.f;
            k += 1.f;
        }
        d1[a] = nd;
        kout[a] = (int)k;
    }
    if (!ok) return false;
    float qw = r.q * w;
    float coef[3];
#pragma unroll
    for (int a = 0; a < DIM; ++a) coef[a] = -qw * r.d[a] / r.dt;
    esirkepov<DIM, P>(acc, cr, d, kout, d1, coef, qw * u[2] * ig);
#pragma unroll
    for (int a = 0; a < DIM; ++a) d[a] = d1[a];
    return true;
}

// Slow path kept out of line so that the staged fast path gets the registers.
template <int DIM, int P>
__device__ __noinline__ bool advance_global(const Run &r, const GlobalFields &gf, const GlobalAcc &gacc, const int *c,
                                            float *d, float *u, float w, int *k)
{
    return advance<DIM, P>(r, gf, gacc, c, d, u, w, k);
}

template <int DIM, int P>
__global__ void __launch_bounds__(256) push_kernel(const Run *__restrict__ runs, const Item *__restrict__ items,
                                                   int tail_block)
{
    extern __shared__ float smem[];
    __shared__ Run rs;
    __shared__ unsigned slow_cnt;
    const Item it = items[blockIdx.x];
    {
        const int *src = reinterpret_cast<const int *>(runs + it.run);
        int *dst = reinterpret_cast<int *>(&rs);
        for (int q = threadIdx.x; q < (int)(sizeof(Run) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
        if (threadIdx.x == 0) slow_cnt = 0;
    }
    __syncthreads();
    const Run &r = rs;
    RunState *stp = r.state;
    const int buf = stp->buf;
    const int origin = stp->origin;
    const long long n_sorted = stp->n_sorted, n_total = stp->n_total;
    const ParticleBuf pb = r.P[buf];
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1;
    const int nl = r.n[DIM - 1];

    long long p0, p1;
    int org[3] = {0, 0, 0}, T[3] = {1, 1, 1};
    const int D = r.drift;
    const bool tile_item = it.kind == 0;
    if (tile_item) {
        const int t = it.a;
        p0 = r.tile_off[t];
        p1 = r.tile_off[t + 1];
        org[0] = (t % r.nt[0]) << r.tlog[0];
        org[1] = ((t / r.nt[0]) % r.nt[1]) << r.tlog[1];
        if (DIM == 3) org[2] = (t / (r.nt[0] * r.nt[1])) << r.tlog[2];
        for (int a = 0; a < DIM; ++a) T[a] = 1 << r.tlog[a];
    } else {
        p0 = n_sorted + (long long)it.a * tail_block;
        p1 = p0 + tail_block < n_total ? p0 + tail_block : n_total;
    }
    if (p0 >= p1) return;

    // shared-memory geometry (tile items only)
    int fh[3] = {0, 0, 0}, fs[3] = {1, 1, 1}, jh[3] = {0, 0, 0}, js[3] = {1, 1, 1};
    for (int a = 0; a < DIM; ++a) {
        fh[a] = D + Reach<P>::GLO;
        fs[a] = T[a] + 2 * D + Reach<P>::GLO + Reach<P>::GHI;
        jh[a] = D + Reach<P>::DLO;
        js[a] = T[a] + 2 * D + Reach<P>::DLO + Reach<P>::DHI;
    }
    const int fvol = fs[0] * fs[1] * fs[2], jvol = js[0] * js[1] * js[2];
    float *Fs = smem;
    float *Js = smem + 6 * fvol;
    if (tile_item) {
        const float *src[6] = {r.E[0], r.E[1], r.E[2], r.B[0], r.B[1], r.B[2]};
        for (int q = threadIdx.x; q < 6 * fvol; q += blockDim.x) {
            int comp = q / fvol, l = q - comp * fvol;
            int lx = l % fs[0], ly = (l / fs[0]) % fs[1], lz = l / (fs[0] * fs[1]);
            int gx = modi(org[0] - fh[0] + lx, n0);
            int gy = modi(org[1] - fh[1] + ly, n1);
            int gz = DIM == 3 ? modi(org[2] - fh[2] + lz, n2) : 0;
            Fs[q] = __ldg(src[comp] + gx + n0 * (gy + n1 * gz));
        }
        for (int q = threadIdx.x; q < 3 * jvol; q += blockDim.x) Js[q] = 0.f;
        __syncthreads();
    }

    const SmemFields sf{Fs, fvol, fh[0], fh[1], fh[2], fs[0], fs[0] * fs[1]};
    const GlobalFields gf{{r.E[0], r.E[1], r.E[2], r.B[0], r.B[1], r.B[2]}, n0, n1, n2};
    const SmemAcc sacc{Js, jvol, jh[0], jh[1], jh[2], js[0], js[0] * js[1]};
    const GlobalAcc gacc{r.J[0], r.J[1], r.J[2], n0, n1, n2};
    unsigned my_slow = 0;

    for (long long i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        int32_t pc = pb.cell[i];
        if (pc < 0) continue;
        int c[3];
        unpack_cell(r, pc, c[0], c[1], c[2]);
        if (r.open_last) {
            int pl = c[DIM - 1] - origin;
            pl = pl < 0 ? pl + nl : pl;
            if (pl < r.margin || pl >= nl - r.margin) {  // left the window: absorbed
                pb.cell[i] = -1;
                continue;
            }
        }
        float d[DIM], u[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) d[a] = pb.off[a][i];
        u[0] = pb.u[0][i];
        u[1] = pb.u[1][i];
        u[2] = pb.u[2][i];
        const float w = pb.w ? pb.w[i] : r.w_const;
        bool fast = tile_item;
        int rel[DIM];
        if (tile_item) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                int v = c[a] - org[a];
                if (v < -D) v += r.n[a];
                else if (v >= T[a] + D) v -= r.n[a];
                rel[a] = v;
                fast = fast && v >= -D && v < T[a] + D;
            }
        }
        int k[DIM];
        bool ok;
        if (fast) {
            ok = advance<DIM, P>(r, sf, sacc, rel, d, u, w, k);
        } else {
            ++my_slow;
            ok = advance_global<DIM, P>(r, gf, gacc, c, d, u, w, k);
        }
        if (!ok) {  // non-finite or over-long move: drop the particle, latch the status
            pb.cell[i] = -1;
            atomicOr(&stp->status, kStatusBadIndex);
            continue;
        }
        // new cell, wrapped (periodic axes and the ring-buffered open axis)
        bool absorbed = false;
#pragma unroll
        for (int a = 0; a < DIM; ++a) c[a] = wrapi(c[a] + k[a], r.n[a]);
        if (r.open_last) {
            int pl = c[DIM - 1] - origin;
            pl = pl < 0 ? pl + nl : pl;
            absorbed = pl < r.margin || pl >= nl - r.margin;
        }
        pb.cell[i] = absorbed ? -1 : pack_cell(r, c[0], c[1], DIM == 3 ? c[2] : 0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) pb.off[a][i] = d[a];
        pb.u[0][i] = u[0];
        pb.u[1][i] = u[1];
        pb.u[2][i] = u[2];
    }
    if (my_slow) atomicAdd(&slow_cnt, my_slow);
    if (tile_item) {
        __syncthreads();
        // flush the tile's current to global J (wrapping the halo)
        float *dst[3] = {r.J[0], r.J[1], r.J[2]};
        for (int q = threadIdx.x; q < 3 * jvol; q += blockDim.x) {
            float v = Js[q];
            if (v == 0.f) continue;
            int comp = q / jvol, l = q - comp * jvol;
            int lx = l % js[0], ly = (l / js[0]) % js[1], lz = l / (js[0] * js[1]);
            int gx = modi(org[0] - jh[0] + lx, n0);
            int gy = modi(org[1] - jh[1] + ly, n1);
            int gz = DIM == 3 ? modi(org[2] - jh[2] + lz, n2) : 0;
            atomicAdd(dst[comp] + gx + n0 * (gy + n1 * gz), v);
        }
    } else {
        __syncthreads();
    }
    if (threadIdx.x == 0 && slow_cnt) atomicAdd(&stp->slow, (unsigned long long)slow_cnt);
}

template <int DIM, int P>
cudaError_t launch_push_t(const Run *runs, const Item *items, int nitems, size_t smem, int block,
                          int tail_block, cudaStream_t st)
{
    auto k = push_kernel<DIM, P>;
    static size_t attr_bytes = 0;  // raise the opt-in shared-memory limit once per size
    if (smem > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    if (nitems == 0) return cudaSuccess;
    k<<<nitems, block, smem, st>>>(runs, items, tail_block);
    return cudaGetLastError();
}

}  // namespace

size_t push_smem_bytes(int dim, int order, const int *tile, int drift)
{
    int glo = 0, ghi = 0, dlo = 0, dhi = 0;
    switch (order) {
    case 1: glo = Reach<1>::GLO; ghi = Reach<1>::GHI; dlo = Reach<1>::DLO; dhi = Reach<1>::DHI; break;
    case 2: glo = Reach<2>::GLO; ghi = Reach<2>::GHI; dlo = Reach<2>::DLO; dhi = Reach<2>::DHI; break;
    default: glo = Reach<3>::GLO; ghi = Reach<3>::GHI; dlo = Reach<3>::DLO; dhi = Reach<3>::DHI; break;
    }
    size_t fv = 1, jv = 1;
    for (int a = 0; a < dim; ++a) {
        fv *= (size_t)(tile[a] + 2 * drift + glo + ghi);
        jv *= (size_t)(tile[a] + 2 * drift + dlo + dhi);
    }
    return sizeof(float) * (6 * fv + 3 * jv);
}

cudaError_t launch_push(int dim, int order, const Run *runs, const Item *items, int nitems, size_t smem,
                        int block, int tail_block, cudaStream_t st)
{
    if (dim == 2) {
        if (order == 1) return launch_push_t<2, 1>(runs, items, nitems, smem, block, tail_block, st);
        if (order == 2) return launch_push_t<2, 2>(runs, items, nitems, smem, block, tail_block, st);
        return launch_push_t<2, 3>(runs, items, nitems, smem, block, tail_block, st);
    }
    if (order == 1) return launch_push_t<3, 1>(runs, items, nitems, smem, block, tail_block, st);
    if (order == 2) return launch_push_t<3, 2>(runs, items, nitems, smem, block, tail_block, st);
    return launch_push_t<3, 3>(runs, items, nitems, smem, block, tail_block, st);
}

}  // namespace pic
