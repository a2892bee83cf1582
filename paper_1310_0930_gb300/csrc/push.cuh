// push.cuh -- fused particle kernel of the EM-PIC timestep (Sec. 5.2 steps
// i-v): per particle, B-spline weights -> gather of E and B at the Yee
// locations -> relativistic Boris push -> move on (cell, offset) -> Esirkepov
// charge-conserving current deposit.
//
// One CTA per tile (a block of TX x TY x TZ cells).  The tile's E and B plus
// a halo are staged in shared memory; its particles (sorted by tile) are
// loaded coalesced from the structure-of-arrays buffers with the next
// particle prefetched; the current of the whole tile is accumulated in a
// shared-memory J tile (the GPU form of the paper's per-thread current
// copies, Sec. 3.1) and flushed to global J once with atomics (the paper's
// reduction of the copies).
//
// The J tile holds each value as two int32 words (hi, lo) of a fixed-point
// number with a per-tile scale S = min(2^30 / (1.01 sum |q w|),
// 4e6 / max |q w|): every single contribution c satisfies
// |c| <= |q w| |v| <= |q w|, so |sum hi| < 2^31 and every scaled
// contribution is below 2^22 in magnitude; lo carries 12 more bits of the
// remainder.  Native int32 shared-memory atomics replace FP32 ones (which
// the hardware emulates with a compare-and-swap loop), integer sums are
// order-independent, and the resolution (2^-42 of the tile's total |q w|
// for tiles of 256 or more equal-weight particles) is finer than FP32
// rounding of the per-node sums.  Because scaled values stay below 2^22,
// both words are rounded to integers by the floating-point add of
// 1.5 * 2^23 (which leaves round-to-nearest(v) in the low mantissa bits)
// instead of conversion instructions.
//
// Tile geometry and the drift allowance are template parameters, so every
// shared-memory address in a particle's stencil is a base register plus an
// immediate offset.  A particle that strayed further than D cells out of
// its tile since the last sort, and every particle of the unsorted tail
// (freshly injected plasma), takes the slow path: the same arithmetic on
// global memory with FP32 global atomics.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace pic {
namespace push_detail {

constexpr float kLoScale = 4096.f;  // 12 bits for the lo word
constexpr float kRound = 12582912.f;  // 1.5 * 2^23: v + kRound = 2^23 + 2^22 + rint(v) for |v| < 2^22
constexpr int kRoundBits = 0x4B400000;  // bit pattern of kRound
constexpr float kMaxScaled = 4.0e6f;  // bound on one scaled contribution (< 2^22, with margin)
constexpr int kTmaSpin = 1 << 20;     // bounded waits on the field-tile barrier
constexpr size_t kSmemBudget = 230000;  // dynamic shared memory of one push CTA (of 227 KB)

// ---------------------------------------------------------------- TMA staging
// The 3D field tile is loaded by the tensor-memory accelerator: one 3D box
// (FX x FY x FZ values) per component into its 128-byte aligned region of
// the shared-memory tile, all six completing on one mbarrier.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmap_acquire(const void *tmap)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

// box at (x, y, z) of the field described by tmap into shared memory dst
__device__ __forceinline__ void tma_load_box(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Kernel variants (template parameter V): the field tile staged by plain
// loads (0) or by TMA (1); 2: plain staging, current deposited as virtual
// trajectories (deposit_split).
constexpr int kVarPlain = 0, kVarTma = 1, kVarSplit = 2;

template <int DIM, int P, int TX, int TY, int TZ, int D, int V>
struct Geo {
    static constexpr int GLO = Reach<P>::GLO, GHI = Reach<P>::GHI, DLO = Reach<P>::DLO, DHI = Reach<P>::DHI;
    static constexpr int up4(int a) { return (a + 3) / 4 * 4; }
    // 3D plane strides padded to 8 or 24 (mod 32) words, whichever needs
    // less padding: stencil rows one plane apart then fall in different
    // shared-memory banks (4 consecutive planes cover 4 distinct bank groups).
    static constexpr int plane(int a)
    {
        return DIM == 3 ? a + ((8 - a % 32 + 32) % 32 < (24 - a % 32 + 32) % 32 ? (8 - a % 32 + 32) % 32
                                                                                : (24 - a % 32 + 32) % 32)
                        : a;
    }
    // J tile: the deposit window of every particle within D cells of the tile
    static constexpr int JX = TX + 2 * D + DLO + DHI, JY = TY + 2 * D + DLO + DHI;
    static constexpr int JZ = DIM == 3 ? TZ + 2 * D + DLO + DHI : 1;
    static constexpr int JHX = D + DLO, JHY = D + DLO, JHZ = DIM == 3 ? D + DLO : 0;
    static constexpr int JPL = plane(JX * JY), JVOL = JPL * JZ;
    // Field tile: rows of FX values starting FHX cells before the tile.
    // T (the TMA layout, 3D): FHX and FX are multiples of 4 so that each row
    // is a TMA box row that starts on a 16-byte boundary of the global field
    // (tile origins are multiples of 8), and the box rows per plane (FY, at
    // least the rows the stencil needs) and FX are chosen so that the dense
    // box planes are 8 or 24 (mod 32) words apart and rows not 0 or 16: a
    // pair whose tile would not fit next to the J tile is skipped; with none
    // left the rows stay dense.  Otherwise: the rows the stencil needs, with
    // 3D planes padded as for the J tile.
    static constexpr bool TL = V == kVarTma && DIM == 3;
    static constexpr bool SPLIT = V == kVarSplit;
    static constexpr int FHX = TL ? up4(D + GLO) : D + GLO, FHY = D + GLO, FHZ = DIM == 3 ? D + GLO : 0;
    static constexpr int FZ = DIM == 3 ? TZ + 2 * D + GLO + GHI : 1;
    static constexpr int NX = TL ? up4(FHX + TX + D + GHI) : TX + 2 * D + GLO + GHI, NY = TY + 2 * D + GLO + GHI;
    static constexpr size_t bytes_for(int bx, int by)
    {
        return 128 + sizeof(float) * 6 * ((bx * by * FZ + 31) / 32 * 32) + sizeof(int) * 6 * JVOL;
    }
    static constexpr bool good(int bx, int by)
    {
        return ((bx * by) % 32 == 8 || (bx * by) % 32 == 24) && bx % 32 != 0 && bx % 32 != 16 &&
               bytes_for(bx, by) <= kSmemBudget;
    }
    static constexpr int pick(int which)
    {
        int best_x = NX, best_y = NY, best = 1 << 30;
        for (int bx = NX; bx <= NX + 16; bx += 4)
            for (int by = NY; by <= NY + 4; ++by)
                if (good(bx, by) && bx * by < best) {
                    best = bx * by;
                    best_x = bx;
                    best_y = by;
                }
        return which == 0 ? best_x : best_y;
    }
    static constexpr int FX = TL ? pick(0) : NX;
    static constexpr int FY = TL ? pick(1) : NY;
    // (the TMA layout keeps dense planes: it is one TMA box per component)
    static constexpr int FPL = TL ? FX * FY : plane(FX * FY);
    // component regions of the field tile start on 128-byte boundaries
    static constexpr int FVOL = (FPL * FZ + 31) / 32 * 32;
    static constexpr unsigned TMA_BYTES = 6u * FZ * FY * FX * sizeof(float);  // one tile, six components
    static __host__ __device__ constexpr int tile(int a) { return a == 0 ? TX : (a == 1 ? TY : (DIM == 3 ? TZ : 1)); }
    // (+128: the field tile is placed at the first 128-byte boundary of the
    // dynamic shared memory, as TMA destinations require)
    static constexpr size_t SMEM_TILES = 128 + sizeof(float) * 6 * FVOL + sizeof(int) * 2 * 3 * JVOL;
    // Deposit staging of one round's moving particles (bucketed deposit, see
    // deposit_round): STG_W words per particle, one padding word per 32 slots.
    static constexpr int STG_W = 8, STG_N = 512 + 512 / 32;
    static constexpr size_t STG_BYTES = sizeof(int) * STG_W * STG_N;
    // The staging is used from quadratic order up, where it fits next to the
    // tiles and the kernel's static shared memory; otherwise each thread
    // deposits its own particle.  Shared-memory atomics of a warp on one
    // address with different values are serialised like a bank conflict, so
    // the lanes that share a row of cells (the sort's order, which makes the
    // gather's loads broadcasts) must not deposit together; dealt by bank the
    // round's atomics are conflict-free.  Measured with row-ordered tiles
    // (256^3 warm plasma, 8 ppc): quadratic push 18.4 -> 15.8 ms, 3D LWFA
    // steps 445-500 32.3 -> 25.7 ms per step; cubic 47.5 -> 30.6 ms before
    // row ordering.
    static constexpr bool BK = P >= 2 && !SPLIT && SMEM_TILES + STG_BYTES + 2048 <= 232448;
    static constexpr size_t SMEM = SMEM_TILES + (BK ? STG_BYTES : 0);
};

// ---------------------------------------------------------------- gather
// Component C from shared memory: bases relative to the tile origin.
template <int DIM, int P, class G, int C>
__device__ __forceinline__ float gather_s(const float *Fs, int bx, int by, int bz, const float *wx,
                                          const float *wy, const float *wz)
{
    const float *p = Fs + C * G::FVOL + (bx + G::FHX) + G::FX * (by + G::FHY) + G::FPL * (bz + G::FHZ);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? P + 1 : 1); ++c) {
        float sy = 0.f;
#pragma unroll
        for (int b = 0; b <= P; ++b) {
            float sx = 0.f;
#pragma unroll
            for (int a = 0; a <= P; ++a) sx = fmaf(wx[a], p[a + G::FX * b + G::FPL * c], sx);
            sy = fmaf(wy[b], sx, sy);
        }
        s = DIM == 3 ? fmaf(wz[c], sy, s) : sy;
    }
    return s;
}

// Component C from global memory, absolute bases wrapped periodically.
struct GlobalFields {
    const float *p[6];
    int n0, n1, n2;
};

template <int DIM, int P, int C>
__device__ __forceinline__ float gather_g(const GlobalFields &g, int bx, int by, int bz, const float *wx,
                                          const float *wy, const float *wz)
{
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? P + 1 : 1); ++c) {
        const int z = DIM == 3 ? wrapi(bz + c, g.n2) : 0;
        float sy = 0.f;
#pragma unroll
        for (int b = 0; b <= P; ++b) {
            const int y = wrapi(by + b, g.n1);
            const float *row = g.p[C] + g.n0 * (y + g.n1 * z);
            float sx = 0.f;
#pragma unroll
            for (int a = 0; a <= P; ++a) sx = fmaf(wx[a], __ldg(row + wrapi(bx + a, g.n0)), sx);
            sy = fmaf(wy[b], sx, sy);
        }
        s = DIM == 3 ? fmaf(wz[c], sy, s) : sy;
    }
    return s;
}

// Relativistic Boris push (Sec. 5.2 step iii): half electric kick, rotation
// with t = (q dt / 2 m gamma) B and s = 2t/(1+t^2), half electric kick.
__device__ __forceinline__ void boris(float h, const float *e, const float *b, float *u)
{
    float um0 = fmaf(h, e[0], u[0]), um1 = fmaf(h, e[1], u[1]), um2 = fmaf(h, e[2], u[2]);
    float ig = rsqrtf(1.f + um0 * um0 + um1 * um1 + um2 * um2);
    float t0 = h * b[0] * ig, t1 = h * b[1] * ig, t2 = h * b[2] * ig;
    float f = 2.f * __frcp_rn(1.f + t0 * t0 + t1 * t1 + t2 * t2);
    float s0 = f * t0, s1 = f * t1, s2 = f * t2;
    float p0 = um0 + (um1 * t2 - um2 * t1);
    float p1 = um1 + (um2 * t0 - um0 * t2);
    float p2 = um2 + (um0 * t1 - um1 * t0);
    u[0] = fmaf(h, e[0], um0 + (p1 * s2 - p2 * s1));
    u[1] = fmaf(h, e[1], um1 + (p2 * s0 - p0 * s2));
    u[2] = fmaf(h, e[2], um2 + (p0 * s1 - p1 * s0));
}

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

// Per-axis Esirkepov window of one straight move: old and new node shapes
// on a (P+2)-node window starting at wb, DS = S1 - S0, A = S0 + DS/2, and
// the prefix sums of DS scaled by coef (the J_a values along a).  When the
// nearest node did not change (shift 0) the last window node carries no
// weight and the last prefix is exactly zero (charge conservation); it is
// set to zero rather than to its rounding residue.
template <int P>
struct Axis {
    float A[P + 2], DS[P + 2], Pre[P + 1];
    int wb;
    int shift;
};

template <int P>
__device__ __forceinline__ void axis_window(int c0, float d0, int k, float d1, float coef, Axis<P> &ax)
{
    int bo, bn;
    float so[P + 1], sn[P + 1], S0[P + 2], S1[P + 2];
    Shape<P>::node(c0, d0, bo, so);
    Shape<P>::node(c0 + k, d1, bn, sn);
    const int s = bn - bo;  // -1, 0 or +1 for a move of less than one cell
    ax.shift = s;
    ax.wb = s < 0 ? bn : bo;
    place<P>(so, s < 0 ? 1 : 0, S0);
    place<P>(sn, s > 0 ? 1 : 0, S1);
    float run = 0.f;
#pragma unroll
    for (int q = 0; q < P + 2; ++q) {
        ax.DS[q] = S1[q] - S0[q];
        ax.A[q] = S0[q] + 0.5f * ax.DS[q];
        if (q < P + 1) {
            run += ax.DS[q];
            ax.Pre[q] = coef * run;
        }
    }
    if (s == 0) ax.Pre[P] = 0.f;
}

// ---------------------------------------------------------------- virtual trajectories
// Sec. 5.2 step iv: the straight move is cut into up to DIM + 1 pieces where
// it crosses a boundary between the grid points nearest the particle (the
// half-integer positions for even orders, the cell faces for odd ones), and
// each piece, which stays with one nearest point per axis, is deposited as a
// move of its own.  Points are kept as (cell, offset) per axis so that the
// move's own end points and the crossing points (exactly 1/2 or 0 from a
// cell) carry no rounding; the other axes' coordinates at a crossing are
// interpolated once and shared by the two pieces that meet there.

// Shape weights of the P + 1 window nodes of a fixed window, tau = the
// position minus the window's reference node: in [-1/2, 1/2] for even
// orders (the middle node), in [0, 1] for odd ones (the cell's lower node).
template <int P>
__device__ __forceinline__ void weights_at(float tau, float *w);
template <>
__device__ __forceinline__ void weights_at<1>(float tau, float *w)
{
    tau = fminf(fmaxf(tau, 0.f), 1.f);
    w[0] = 1.f - tau;
    w[1] = tau;
}
template <>
__device__ __forceinline__ void weights_at<2>(float tau, float *w)
{
    Shape<2>::q(fminf(fmaxf(tau, -0.5f), 0.5f), w);
}
template <>
__device__ __forceinline__ void weights_at<3>(float tau, float *w)
{
    Shape<3>::cub(fminf(fmaxf(tau, 0.f), 1.f), w);
}
template <>
__device__ __forceinline__ void weights_at<4>(float tau, float *w)
{
    Shape<4>::q(fminf(fmaxf(tau, -0.5f), 0.5f), w);
}

// reference node of a point (cell c, offset o): the nearest integer for even
// orders, the cell for odd ones
template <int P>
__device__ __forceinline__ int ref_node(int c, float o)
{
    return P % 2 == 0 ? c + (o >= 0.5f ? 1 : 0) : c;
}

// Cut the move (c[a], d0[a]) -> (c[a] + k[a], d1[a]) into pieces and call
// piece(ax, frac) for each, ax the piece's no-shift Esirkepov windows
// (coef_a = -q w d_a / dt) and frac its share of the time step.
template <int DIM, int P, class Piece>
__device__ __forceinline__ void split_move(const int *c, const float *d0, const int *k, const float *d1,
                                           const float *coef, const Piece &piece)
{
    float tcut[DIM] = {};
    int acut[DIM] = {}, ncut = 0;
    int n0[DIM], n1[DIM], bc[DIM];
    float bo[DIM], dx[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        n0[a] = ref_node<P>(c[a], d0[a]);
        n1[a] = ref_node<P>(c[a] + k[a], d1[a]);
        dx[a] = ((float)k[a] + d1[a]) - d0[a];  // displacement in cells
        bc[a] = c[a];
        bo[a] = d0[a];
        if (n1[a] != n0[a]) {  // crossing: the boundary as (cell, offset)
            const int s = n1[a] - n0[a];
            if (P % 2 == 0) {
                bc[a] = s > 0 ? n0[a] : n0[a] - 1;
                bo[a] = 0.5f;
            } else {
                bc[a] = s > 0 ? n0[a] + 1 : n0[a];
                bo[a] = 0.f;
            }
            tcut[ncut] = (((float)(bc[a] - c[a]) + bo[a]) - d0[a]) / dx[a];
            acut[ncut] = a;
            ++ncut;
        }
    }
#pragma unroll
    for (int i = 1; i < DIM; ++i)  // ascending (at most DIM cuts)
#pragma unroll
        for (int j = DIM - 1; j >= 1; --j)
            if (j < ncut && tcut[j] < tcut[j - 1]) {
                const float t = tcut[j];
                tcut[j] = tcut[j - 1];
                tcut[j - 1] = t;
                const int q = acut[j];
                acut[j] = acut[j - 1];
                acut[j - 1] = q;
            }
    int sc[DIM];  // start point of the current piece
    float so[DIM];
    unsigned done = 0;  // bit a: the axis was crossed before the current piece
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        sc[a] = c[a];
        so[a] = d0[a];
    }
    float t0 = 0.f;
    // (the remaining cuts are kept in tcut[0..], acut[0..]: shifted down after
    // each piece, so that every index is a compile-time constant)
    for (int i = 0; i <= ncut; ++i) {
        const bool last = i == ncut;
        const float t1 = last ? 1.f : tcut[0];
        const int cut_axis = last ? -1 : acut[0];
        int ec[DIM];
        float eo[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            if (last) {
                ec[a] = c[a] + k[a];
                eo[a] = d1[a];
            } else if (a == cut_axis) {
                ec[a] = bc[a];
                eo[a] = bo[a];
            } else {
                const float o = d0[a] + t1 * dx[a];
                const float f = floorf(o);
                ec[a] = c[a] + (int)f;
                eo[a] = o - f;
                if (eo[a] >= 1.f) {
                    eo[a] = 0.f;
                    ec[a] += 1;
                }
            }
        }
        Axis<P> ax[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int node = ((done >> a) & 1u) ? n1[a] : n0[a];
            float S0[P + 1], S1[P + 1];
            weights_at<P>((float)(sc[a] - node) + so[a], S0);
            weights_at<P>((float)(ec[a] - node) + eo[a], S1);
            ax[a].wb = node - P / 2;
            ax[a].shift = 0;
            float run = 0.f;
#pragma unroll
            for (int q = 0; q < P + 2; ++q) {
                const float s0 = q <= P ? S0[q] : 0.f, s1 = q <= P ? S1[q] : 0.f;
                ax[a].DS[q] = s1 - s0;
                ax[a].A[q] = s0 + 0.5f * ax[a].DS[q];
                if (q < P + 1) {
                    run += ax[a].DS[q];
                    ax[a].Pre[q] = coef[a] * run;
                }
            }
            ax[a].Pre[P] = 0.f;  // (the window's total change is zero)
        }
        piece(reinterpret_cast<const Axis<P> *>(ax), t1 - t0);
        if (!last) done |= 1u << cut_axis;
#pragma unroll
        for (int j = 0; j + 1 < DIM; ++j) {
            tcut[j] = tcut[j + 1];
            acut[j] = acut[j + 1];
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            sc[a] = ec[a];
            so[a] = eo[a];
        }
        t0 = t1;
    }
}

// Esirkepov deposit (Sec. 5.2 charge-conserving deposit):
//   3D: J_a(window) = coef_a * prefix_a(DS_a) * (A_b A_c + DS_b DS_c / 12),
//   2D: J_x = coef_x prefix_x(DS_x) A_y, J_y = coef_y prefix_y(DS_y) A_x,
//       J_z = q w v_z (A_x A_y + DS_x DS_y / 12),
// coef_a = -q w d_a / dt.  (A_b A_c + DS_b DS_c/12 equals the textbook
// S0S0 + DS S0/2 + S0 DS/2 + DS DS/3.)  `emit(comp, qa, qb, qc, v)` receives
// each value with its window coordinates (axis order x, y, z).
template <int DIM, int P, class Emit>
__device__ __forceinline__ void esirkepov(const Axis<P> *ax, float qwvz, const Emit &emit)
{
    constexpr int W = P + 2;
    const float twelfth = 1.f / 12.f;
    if (DIM == 3) {
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const int a = comp, b = (comp + 1) % 3, c = (comp + 2) % 3;
#pragma unroll
            for (int qc = 0; qc < W; ++qc)
#pragma unroll
                for (int qb = 0; qb < W; ++qb) {
                    const float fac = fmaf(ax[b].DS[qb] * twelfth, ax[c].DS[qc], ax[b].A[qb] * ax[c].A[qc]);
#pragma unroll
                    for (int qa = 0; qa < W - 1; ++qa) {
                        int q3[3];
                        q3[a] = qa;
                        q3[b] = qb;
                        q3[c] = qc;
                        emit(comp, q3[0], q3[1], q3[2], ax[a].Pre[qa] * fac);
                    }
                }
        }
    } else {
#pragma unroll
        for (int qb = 0; qb < W; ++qb)
#pragma unroll
            for (int qa = 0; qa < W; ++qa) {
                if (qa < W - 1) emit(0, qa, qb, 0, ax[0].Pre[qa] * ax[1].A[qb]);
                if (qb < W - 1) emit(1, qa, qb, 0, ax[1].Pre[qb] * ax[0].A[qa]);
                emit(2, qa, qb, 0,
                     qwvz * fmaf(ax[0].DS[qa] * twelfth, ax[1].DS[qb], ax[0].A[qa] * ax[1].A[qb]));
            }
    }
}

// One particle's weights, gather, push and move.  cr: cell coordinates in
// the accessor's frame.  live = false (uniform over the CTA) says that every
// field value the gather could read is +0, so the interpolated E and B are +0
// exactly and the weights and the gather are skipped.  Returns false for a
// non-finite or over-long move.
template <int DIM, int P, class GatherFn>
__device__ __forceinline__ bool push_move(const Run &r, const GatherFn &gather, const int *cr, const float *d,
                                          float *u, float *d1, int *k, float &ig, bool live = true)
{
    float e[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
    if (live) {
        int bn[3] = {0, 0, 0}, bh[3] = {0, 0, 0};
        float wn[3][P + 1], wh[3][P + 1];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            Shape<P>::node(cr[a], d[a], bn[a], wn[a]);
            Shape<P>::half(cr[a], d[a], bh[a], wh[a]);
        }
        if (DIM == 2) {
#pragma unroll
            for (int q = 0; q <= P; ++q) wn[2][q] = wh[2][q] = 0.f;
        }
        gather(bn, bh, wn, wh, e, b);
    }
    boris(r.qm_half_dt, e, b, u);
    ig = rsqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        float nd = d[a] + r.dt_over_d[a] * u[a] * ig;
        ok = ok && nd > -1.f && nd < 2.f;  // false for NaN too
        nd = ok ? nd : d[a];
        float kk = floorf(nd);
        nd = nd - kk;
        if (nd >= 1.f) {  // FP32 rounding of a value just below an integer
            nd = 0.f;
            kk += 1.f;
        }
        d1[a] = nd;
        k[a] = (int)kk;
    }
    return ok;
}

// Yee locations: E0 (h,n,n) E1 (n,h,n) E2 (n,n,h) B0 (n,h,h) B1 (h,n,h) B2 (h,h,n);
// h = half-integer, n = integer; bit c of kHalf{X,Y,Z} marks component c as
// half-integer along that axis.  In 2D the third entry is unused.
constexpr unsigned kHalfX = 0x31u, kHalfY = 0x2Au, kHalfZ = 0x1Cu;

// Shared-memory gather of the six components; each component's loads are
// immediate offsets from one base address.
template <int DIM, int P, class G>
struct SmemGather {
    const float *Fs;
    __device__ __forceinline__ void operator()(const int *bn, const int *bh, const float (*wn)[P + 1],
                                               const float (*wh)[P + 1], float *e, float *b) const
    {
        e[0] = gather_s<DIM, P, G, 0>(Fs, bh[0], bn[1], bn[2], wh[0], wn[1], wn[2]);
        e[1] = gather_s<DIM, P, G, 1>(Fs, bn[0], bh[1], bn[2], wn[0], wh[1], wn[2]);
        e[2] = gather_s<DIM, P, G, 2>(Fs, bn[0], bn[1], bh[2], wn[0], wn[1], wh[2]);
        b[0] = gather_s<DIM, P, G, 3>(Fs, bn[0], bh[1], bh[2], wn[0], wh[1], wh[2]);
        b[1] = gather_s<DIM, P, G, 4>(Fs, bh[0], bn[1], bh[2], wh[0], wn[1], wh[2]);
        b[2] = gather_s<DIM, P, G, 5>(Fs, bh[0], bh[1], bn[2], wh[0], wh[1], wn[2]);
    }
};

// Add one value to the fixed-point J tile at hi (its lo word JLO words
// further): x = ps * fac (ps already scaled by S, |x| < 2^22) split into the
// integer nearest to the exact product (hi) and 12 bits of the remainder
// (lo).  t = fma(ps, fac, 1.5 * 2^23) holds that integer in its low mantissa
// bits; the remainder fma(ps, fac, -integer) is exact to FP32 rounding of a
// value below 1.  `on` is false where this lane's value is zero by
// structure (the far window node of an axis along which the lane did not
// change nodes); it predicates the two atomics, with no branch per value.
template <int JLO>
__device__ __forceinline__ void fix_add(int *hi, float ps, float fac, bool on)
{
    const float t = fmaf(ps, fac, kRound);          // kRound + rint(x), exact
    const float rem = fmaf(ps, fac, kRound - t);    // x - rint(x), |rem| <= 1/2
    const float tl = fmaf(rem, kLoScale, kRound);
    const int vh = __float_as_int(t) - kRoundBits, vl = __float_as_int(tl) - kRoundBits;
    if (on) {
        atomicAdd(hi, vh);
        atomicAdd(hi + JLO, vl);
    }
}

// 3D Esirkepov deposit into the shared-memory J tile: a loop over the three
// components, axis roles (a, b, c) = (comp, comp+1, comp+2) selected per
// iteration.  Component a has W-1 prefix-sum values along a (qa) and W
// window nodes along b and c; along an axis where the lane kept its nearest
// node the far value (qa = W-2, qb = W-1 or qc = W-1) is zero by structure.
// The near block is added unconditionally; each far face, edge and corner
// the lane needs is one branch (one divergent region per face and lane
// condition, not one per value): for the common case of no node change
// this is 54 values instead of 144.
template <int P, class G>
__device__ __forceinline__ void deposit3_smem(const Axis<P> *ax, float S, int *Jhi)
{
    constexpr int W = P + 2, NA = W - 2, NB = W - 1;  // near values: qa < NA; qb, qc < NB
    constexpr int JLO = 3 * G::JVOL;
    const float twelfth = 1.f / 12.f;
    const bool m0 = ax[0].shift != 0, m1 = ax[1].shift != 0, m2 = ax[2].shift != 0;  // this lane
    const int base = (ax[0].wb + G::JHX) + G::JX * (ax[1].wb + G::JHY) + G::JPL * (ax[2].wb + G::JHZ);
    constexpr int s0 = 1, s1 = G::JX, s2 = G::JPL;
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        float pa[W - 1], Ab[W], Db[W], Ac[W], Dc[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (q < W - 1)
                pa[q] = S * (comp == 0 ? ax[0].Pre[q] : (comp == 1 ? ax[1].Pre[q] : ax[2].Pre[q]));
            Ab[q] = comp == 0 ? ax[1].A[q] : (comp == 1 ? ax[2].A[q] : ax[0].A[q]);
            Db[q] = (comp == 0 ? ax[1].DS[q] : (comp == 1 ? ax[2].DS[q] : ax[0].DS[q])) * twelfth;
            Ac[q] = comp == 0 ? ax[2].A[q] : (comp == 1 ? ax[0].A[q] : ax[1].A[q]);
            Dc[q] = comp == 0 ? ax[2].DS[q] : (comp == 1 ? ax[0].DS[q] : ax[1].DS[q]);
        }
        const int sa = comp == 0 ? s0 : (comp == 1 ? s1 : s2);
        const int sb = comp == 0 ? s1 : (comp == 1 ? s2 : s0);
        const int sc = comp == 0 ? s2 : (comp == 1 ? s0 : s1);
        const bool ma = comp == 0 ? m0 : (comp == 1 ? m1 : m2);
        const bool mb = comp == 0 ? m1 : (comp == 1 ? m2 : m0);
        const bool mc = comp == 0 ? m2 : (comp == 1 ? m0 : m1);
        int *hb = Jhi + comp * G::JVOL + base;
        // near block, then the far a-face of each near c row
#pragma unroll
        for (int qc = 0; qc < NB; ++qc) {
            float f[NB];
#pragma unroll
            for (int qb = 0; qb < NB; ++qb) {
                f[qb] = fmaf(Db[qb], Dc[qc], Ab[qb] * Ac[qc]);
#pragma unroll
                for (int qa = 0; qa < NA; ++qa) fix_add<JLO>(hb + qa * sa + qb * sb + qc * sc, pa[qa], f[qb], true);
            }
            if (ma) {
#pragma unroll
                for (int qb = 0; qb < NB; ++qb) fix_add<JLO>(hb + NA * sa + qb * sb + qc * sc, pa[NA], f[qb], true);
            }
        }
        // far b-face (qb = NB) over the near c rows, and its a-edge
        if (mb) {
            float f[NB];
#pragma unroll
            for (int qc = 0; qc < NB; ++qc) {
                f[qc] = fmaf(Db[NB], Dc[qc], Ab[NB] * Ac[qc]);
#pragma unroll
                for (int qa = 0; qa < NA; ++qa) fix_add<JLO>(hb + qa * sa + NB * sb + qc * sc, pa[qa], f[qc], true);
            }
            if (ma) {
#pragma unroll
                for (int qc = 0; qc < NB; ++qc) fix_add<JLO>(hb + NA * sa + NB * sb + qc * sc, pa[NA], f[qc], true);
            }
        }
        // far c-face (qc = NB) over the near b rows, and its a-edge
        if (mc) {
            float f[NB];
#pragma unroll
            for (int qb = 0; qb < NB; ++qb) {
                f[qb] = fmaf(Db[qb], Dc[NB], Ab[qb] * Ac[NB]);
#pragma unroll
                for (int qa = 0; qa < NA; ++qa) fix_add<JLO>(hb + qa * sa + qb * sb + NB * sc, pa[qa], f[qb], true);
            }
            if (ma) {
#pragma unroll
                for (int qb = 0; qb < NB; ++qb) fix_add<JLO>(hb + NA * sa + qb * sb + NB * sc, pa[NA], f[qb], true);
            }
        }
        // the (b, c) far edge and the corner
        if (mb && mc) {
            const float f = fmaf(Db[NB], Dc[NB], Ab[NB] * Ac[NB]);
#pragma unroll
            for (int qa = 0; qa < NA; ++qa) fix_add<JLO>(hb + qa * sa + NB * sb + NB * sc, pa[qa], f, true);
            if (ma) fix_add<JLO>(hb + NA * sa + NB * sb + NB * sc, pa[NA], f, true);
        }
    }
}

// 2D Esirkepov deposit into the shared-memory J tile (J_x, J_y from the
// in-plane moves, J_z from v_z), same rule: the near block unconditionally,
// the far x values, the far y values and the corner each under one branch.
template <int P, class G>
__device__ __forceinline__ void deposit2_smem(const Axis<P> *ax, float S, float qwvz, int *Jhi)
{
    constexpr int W = P + 2;
    constexpr int JLO = 3 * G::JVOL;
    const float twelfth = 1.f / 12.f;
    const bool m0 = ax[0].shift != 0, m1 = ax[1].shift != 0;
    int *const h0 = Jhi + (ax[0].wb + G::JHX) + G::JX * (ax[1].wb + G::JHY);
    float px[W - 1], py[W - 1];
#pragma unroll
    for (int q = 0; q < W - 1; ++q) {
        px[q] = S * ax[0].Pre[q];
        py[q] = S * ax[1].Pre[q];
    }
    const float sz = S * qwvz;
    // J_x at (qa, qb), qa < W - 1 prefix values; J_y at (qa, qb), qb < W - 1;
    // J_z at every window node
    auto jx = [&](int qa, int qb) { fix_add<JLO>(h0 + qa + G::JX * qb, px[qa], ax[1].A[qb], true); };
    auto jy = [&](int qa, int qb) { fix_add<JLO>(h0 + G::JVOL + qa + G::JX * qb, py[qb], ax[0].A[qa], true); };
    auto jz = [&](int qa, int qb) {
        fix_add<JLO>(h0 + 2 * G::JVOL + qa + G::JX * qb, sz,
                     fmaf(ax[0].DS[qa] * twelfth, ax[1].DS[qb], ax[0].A[qa] * ax[1].A[qb]), true);
    };
#pragma unroll
    for (int qb = 0; qb < W - 1; ++qb) {
#pragma unroll
        for (int qa = 0; qa < W - 1; ++qa) {
            if (qa < W - 2) jx(qa, qb);
            if (qb < W - 2) jy(qa, qb);
            jz(qa, qb);
        }
    }
    if (m0) {  // far x: J_x at qa = W - 2, J_y and J_z at qa = W - 1
#pragma unroll
        for (int qb = 0; qb < W - 1; ++qb) {
            jx(W - 2, qb);
            if (qb < W - 2) jy(W - 1, qb);
            jz(W - 1, qb);
        }
    }
    if (m1) {  // far y: J_y at qb = W - 2, J_x and J_z at qb = W - 1
#pragma unroll
        for (int qa = 0; qa < W - 1; ++qa) {
            if (qa < W - 2) jx(qa, W - 1);
            jy(qa, W - 2);
            jz(qa, W - 1);
        }
    }
    if (m0 && m1) {
        jx(W - 2, W - 1);
        jy(W - 1, W - 2);
        jz(W - 1, W - 1);
    }
}

// Node base of the Esirkepov window of a move from (c, d) by k cells to d1
// along one axis: the lower of the old and new nearest-node bases.
template <int P>
__device__ __forceinline__ int window_base(int c, float d, int k, float d1)
{
    int bo, bn;
    float w[P + 1];
    Shape<P>::node(c, d, bo, w);
    Shape<P>::node(c + k, d1, bn, w);
    return bo < bn ? bo : bn;
}

// Bucketed deposit of one round (all threads of the CTA call it together).
// The current is what the thread-per-particle deposit gives; only the
// assignment of particles to threads changes.  The moving particles of the
// round are sorted by the shared-memory bank of their J window base (a
// counting sort into 32 buckets), then warp w takes the particles w, w + nw,
// w + 2 nw, ... of that order: the lanes of a warp then hold windows in
// (mostly) distinct banks, so the window's atomics, whose offsets from the
// base are the same for every lane, are (mostly) free of bank conflicts.
// A particle that moves is described by its staged record: packed tile
// coordinates and cell carries, old and new offsets, q w and (2D) q w v_z.
// Returns the number of particles of the round that deposited.
template <int DIM, int P, class G>
__device__ __forceinline__ int deposit_round(const Run &r, bool dep, int pk, const float *d0, const float *d1,
                                             float qw, float qwvz, float S, int *Jhi, int *stg, int *s_cnt,
                                             int *s_start)
{
    const unsigned lane = threadIdx.x & 31u;
    int bank = 0;
    if (dep) {
        int wb[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            wb[a] = window_base<P>(((pk >> (8 * a)) & 255) - 64, d0[a], ((pk >> (24 + 2 * a)) & 3) - 1, d1[a]);
        bank = ((wb[0] + G::JHX) + G::JX * (wb[1] + G::JHY) + G::JPL * (wb[2] + G::JHZ)) & 31;
    }
    const unsigned m = __match_any_sync(0xffffffffu, dep ? bank : 32 + (int)lane);
    const int leader = __ffs(m) - 1;
    int b0 = 0;
    if (dep && (int)lane == leader) b0 = atomicAdd(s_cnt + bank, __popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, leader);
    const int rank = b0 + __popc(m & ((1u << lane) - 1u));
    const int ndep = __syncthreads_count(dep);
    if (ndep == 0) return 0;  // (uniform; the counters are all still zero)
    if (threadIdx.x < 32) {  // exclusive scan of the bucket counts
        const int c = s_cnt[lane];
        int v = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if ((int)lane >= o) v += t;
        }
        s_start[lane] = v - c;
    }
    __syncthreads();
    if (threadIdx.x < 32) s_cnt[lane] = 0;  // (next counted after the next barrier)
    if (dep) {
        int q = s_start[bank] + rank;
        q += q >> 5;
        stg[q] = pk;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            stg[(1 + a) * G::STG_N + q] = __float_as_int(d0[a]);
            stg[(1 + DIM + a) * G::STG_N + q] = __float_as_int(d1[a]);
        }
        stg[(1 + 2 * DIM) * G::STG_N + q] = __float_as_int(qw);
        if (DIM == 2) stg[(2 + 2 * DIM) * G::STG_N + q] = __float_as_int(qwvz);
    }
    __syncthreads();
    const int nw = (ndep + 31) >> 5, w = threadIdx.x >> 5;
    int q = (int)lane * nw + w;
    if (w < nw && q < ndep) {
        q += q >> 5;
        const int rpk = stg[q];
        int rel[3], k[3];
        float a0[3], a1[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            rel[a] = ((rpk >> (8 * a)) & 255) - 64;
            k[a] = ((rpk >> (24 + 2 * a)) & 3) - 1;
            a0[a] = __int_as_float(stg[(1 + a) * G::STG_N + q]);
            a1[a] = __int_as_float(stg[(1 + DIM + a) * G::STG_N + q]);
        }
        const float rqw = __int_as_float(stg[(1 + 2 * DIM) * G::STG_N + q]);
        Axis<P> ax[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) axis_window<P>(rel[a], a0[a], k[a], a1[a], -rqw * r.d_over_dt[a], ax[a]);
        if (DIM == 3) deposit3_smem<P, G>(reinterpret_cast<const Axis<P> *>(ax), S, Jhi);
        else
            deposit2_smem<P, G>(reinterpret_cast<const Axis<P> *>(ax), S,
                                __int_as_float(stg[(2 + 2 * DIM) * G::STG_N + q]), Jhi);
    }
    return ndep;
}

template <int DIM, int P>
struct GlobalGather {
    GlobalFields g;
    __device__ __forceinline__ void operator()(const int *bn, const int *bh, const float (*wn)[P + 1],
                                               const float (*wh)[P + 1], float *e, float *b) const
    {
        e[0] = gather_g<DIM, P, 0>(g, bh[0], bn[1], bn[2], wh[0], wn[1], wn[2]);
        e[1] = gather_g<DIM, P, 1>(g, bn[0], bh[1], bn[2], wn[0], wh[1], wn[2]);
        e[2] = gather_g<DIM, P, 2>(g, bn[0], bn[1], bh[2], wn[0], wn[1], wh[2]);
        b[0] = gather_g<DIM, P, 3>(g, bn[0], bh[1], bh[2], wn[0], wh[1], wh[2]);
        b[1] = gather_g<DIM, P, 4>(g, bh[0], bn[1], bh[2], wh[0], wn[1], wh[2]);
        b[2] = gather_g<DIM, P, 5>(g, bh[0], bh[1], bn[2], wh[0], wh[1], wn[2]);
    }
};

struct ParticleIn {
    int32_t cell;
    float off[3];
    float u[3];
    float w;
};

__device__ __forceinline__ void load_particle(const ParticleBuf &pb, int dim, long long i, float w_const,
                                              ParticleIn &p)
{
    p.cell = pb.cell[i];
    p.off[0] = pb.off[0][i];
    p.off[1] = pb.off[1][i];
    p.off[2] = dim == 3 ? pb.off[2][i] : 0.f;
    p.u[0] = pb.u[0][i];
    p.u[1] = pb.u[1][i];
    p.u[2] = pb.u[2][i];
    p.w = pb.w ? pb.w[i] : w_const;
}

struct SlowOut {
    float d[3], u[3];
    int k[3];
    int ok;
};

// Slow path, kept out of line so that the staged fast path gets the
// registers; arguments by value so that no fast-path variable has its
// address taken.
template <int DIM, int P, bool SPLIT = false>
__device__ __noinline__ SlowOut advance_global(const Run &r, const GlobalFields gf, int c0, int c1, int c2, float e0,
                                               float e1, float e2, float u0, float u1, float u2, float w)
{
    SlowOut o;
    const int c[3] = {c0, c1, c2};
    float d[3] = {e0, e1, e2}, u[3] = {u0, u1, u2};
    int k[3] = {0, 0, 0};
    float d1[3] = {0.f, 0.f, 0.f}, ig;
    const GlobalGather<DIM, P> gather{gf};
    o.ok = push_move<DIM, P>(r, gather, c, d, u, d1, k, ig);
    if (!o.ok) return o;
    if (r.jt) {  // this move deposits current near its tile: the tile's neighbours are not quiet
        bool moves = DIM == 2 && u[2] != 0.f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) moves = moves || k[a] != 0 || d1[a] != d[a];
        if (moves) r.jt[tile_of(r, c0, c1, DIM == 3 ? c2 : 0)] = 1;
    }
    const float qw = r.q * w;
    float *J[3] = {r.J[0], r.J[1], r.J[2]};
    const int n0 = gf.n0, n1 = gf.n1, n2 = gf.n2;
    auto deposit = [&](const Axis<P> *ax, float qwvz) {
        esirkepov<DIM, P>(ax, qwvz, [&](int comp, int qa, int qb, int qc, float v) {
            if (v == 0.f) return;
            const int x = wrapi(ax[0].wb + qa, n0), y = wrapi(ax[1].wb + qb, n1);
            const int z = DIM == 3 ? wrapi(ax[DIM - 1].wb + qc, n2) : 0;
            atomicAdd(J[comp] + (long long)(x + n0 * (y + n1 * z)) * r.jst, v);
        });
    };
    if (SPLIT) {
        float coef[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) coef[a] = -qw * r.d_over_dt[a];
        const float qwvz = qw * u[2] * ig;
        split_move<DIM, P>(c, d, k, d1, coef, [&](const Axis<P> *ax, float frac) { deposit(ax, qwvz * frac); });
    } else {
        Axis<P> ax[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) axis_window<P>(c[a], d[a], k[a], d1[a], -qw * r.d_over_dt[a], ax[a]);
        deposit(ax, qw * u[2] * ig);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.d[a] = d1[a];
        o.u[a] = u[a];
        o.k[a] = k[a];
    }
    return o;
}

constexpr int kStage = 6;  // field-tile rows loaded at once per thread

// One work item: a tile of one run (staged fast path) or a block of that
// run's unsorted tail (slow path).  Called uniformly by the whole CTA.
template <int DIM, int P, int TX, int TY, int TZ, int D, int V>
__device__ __forceinline__ void process_item(const Run *__restrict__ runs, const Item it, int tail_block)
{
    using G = Geo<DIM, P, TX, TY, TZ, D, V>;
    extern __shared__ __align__(16) float smem[];
    __shared__ Run rs;
    __shared__ unsigned slow_cnt;
    __shared__ float wsum[32], wmaxs[32];
    __shared__ int s_cnt[32], s_start[32];
    __shared__ __align__(8) uint64_t tma_bar;
    if (G::TL && threadIdx.x == 0) mbar_init(&tma_bar);
    {
        const int *src = reinterpret_cast<const int *>(runs + it.run);
        int *dst = reinterpret_cast<int *>(&rs);
        for (int q = threadIdx.x; q < (int)(sizeof(Run) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
        if (threadIdx.x == 0) slow_cnt = 0;
        if (threadIdx.x < 32) s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    const Run &r = rs;
    RunState *stp = r.state;
    const int origin = stp->origin;
    const long long n_sorted = stp->n_sorted, n_total = stp->n_total;
    const ParticleBuf pb = r.P[stp->buf];
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1;
    const int nl = r.n[DIM - 1];
    const bool tile_item = it.kind == 0;

    long long p0, p1;
    int org[3] = {0, 0, 0};
    if (tile_item) {
        const int t = it.a;
        p0 = r.tile_off[t];
        p1 = r.tile_off[t + 1];
        org[0] = (t % r.nt[0]) * TX;
        org[1] = ((t / r.nt[0]) % r.nt[1]) * TY;
        if (DIM == 3) org[2] = (t / (r.nt[0] * r.nt[1])) * TZ;
    } else {
        p0 = n_sorted + (long long)it.a * tail_block;
        p1 = p0 + tail_block < n_total ? p0 + tail_block : n_total;
    }
    if (p0 >= p1) {
        if (G::TL && threadIdx.x == 0) mbar_inval(&tma_bar);
        return;
    }

    // (an offset from the shared array, so that the compiler keeps shared
    // loads and stores for the tiles)
    float *Fs = smem + ((128u - (smem_addr(smem) & 127u)) & 127u) / sizeof(float);
    int *Jhi = reinterpret_cast<int *>(Fs + 6 * G::FVOL);
    int *Jlo = Jhi + 3 * G::JVOL;
    int *stg = Jlo + 3 * G::JVOL;  // deposit staging (G::BK)
    float S = 1.f;  // fixed-point scale of this tile's J
    // TMA staging: 3D tiles whose field box lies inside the stored grid
    // (boxes that wrap around a periodic or ring boundary are loaded below)
    bool tma = false;
    bool live = true;  // some staged field value is not +0
    if (G::TL && tile_item && r.tmap) {
        const int x0 = org[0] - G::FHX, y0 = org[1] - G::FHY, z0 = org[2] - G::FHZ;
        tma = x0 >= 0 && x0 + G::FX <= n0 && y0 >= 0 && y0 + G::FY <= n1 && z0 >= 0 && z0 + G::FZ <= n2;
        // the box row must start on a 16-byte boundary of the field and each
        // destination on a 128-byte boundary of shared memory
        tma = tma && (x0 & 3) == 0 && (smem_addr(Fs) & 127u) == 0 && ((G::FVOL * sizeof(float)) & 127u) == 0;
        if (tma && threadIdx.x == 0) {
            const char *maps = reinterpret_cast<const char *>(r.tmap);
            mbar_expect(&tma_bar, G::TMA_BYTES);
            for (int c = 0; c < 6; ++c) {
                const void *m = maps + 128 * c;
                tmap_acquire(m);
                tma_load_box(Fs + c * G::FVOL, m, x0, y0, z0, &tma_bar);
            }
        }
    }
    if (tile_item) {
        unsigned nzbits = tma ? 1u : 0u;  // (TMA-staged tiles are taken as live)
        // (kStage rows of loads in flight per thread before their stores)
        for (int l0 = tma ? G::FVOL : threadIdx.x; l0 < G::FVOL; l0 += kStage * blockDim.x) {
            float v[kStage][6];
            int ls[kStage];
#pragma unroll
            for (int s = 0; s < kStage; ++s) {
                const int l = l0 + s * blockDim.x;
                ls[s] = -1;
                if (l < G::FVOL) {
                    const int lz = l / G::FPL, lxy = l - lz * G::FPL, ly = lxy / G::FX, lx = lxy - ly * G::FX;
                    if (ly < G::FY) {  // (else plane padding)
                        const int gx = modi(org[0] - G::FHX + lx, n0);
                        const int gy = modi(org[1] - G::FHY + ly, n1);
                        const int gz = DIM == 3 ? modi(org[2] - G::FHZ + lz, n2) : 0;
                        const int g = gx + n0 * (gy + n1 * gz);
                        ls[s] = l;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            v[s][c] = __ldg(r.E[c] + g);
                            v[s][3 + c] = __ldg(r.B[c] + g);
                        }
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < kStage; ++s)
                if (ls[s] >= 0) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        Fs[c * G::FVOL + ls[s]] = v[s][c];
                        nzbits |= __float_as_uint(v[s][c]);
                    }
                }
        }
        for (int q = threadIdx.x; q < 6 * G::JVOL; q += blockDim.x) Jhi[q] = 0;
        // scale bounds: sum and maximum of |q w| over the tile's particles
        float wtot, wmax;
        if (pb.w) {
            float acc = 0.f, mx = 0.f;
            for (long long i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
                const float a = fabsf(pb.w[i]);
                acc += a;
                mx = fmaxf(mx, a);
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(0xffffffffu, acc, o);
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if ((threadIdx.x & 31) == 0) {
                wsum[threadIdx.x >> 5] = acc;
                wmaxs[threadIdx.x >> 5] = mx;
            }
            __syncthreads();
            wtot = 0.f;
            wmax = 0.f;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                wtot += wsum[q];
                wmax = fmaxf(wmax, wmaxs[q]);
            }
        } else {
            wtot = fabsf(r.w_const) * (float)(p1 - p0);
            wmax = fabsf(r.w_const);
        }
        const float B = 1.01f * fabsf(r.q) * wtot, M = fabsf(r.q) * wmax;
        S = B > 0.f ? fminf(1073741824.f / B, kMaxScaled / M) : 1.f;
        bool done = true;
        if (tma) {  // bounded wait for the field tile; a timeout is latched in the status
            done = false;
            for (int it = 0; it < kTmaSpin && !done; ++it) done = mbar_try_wait(&tma_bar, 0);
            if (!done) {
                if (threadIdx.x == 0) atomicOr(&stp->status, kStatusTimeout);
                for (int it = 0; it < kTmaSpin && !done; ++it) done = mbar_try_wait(&tma_bar, 0);
            }
        }
        // a field tile that did not arrive in time: the whole CTA leaves the
        // tile's particles and current as they are (the latched status reports
        // the incomplete step) rather than push with a partly written tile
        if (__syncthreads_or(!done)) return;
        live = __syncthreads_or(nzbits != 0u) != 0;
    }

    const GlobalFields gf{{r.E[0], r.E[1], r.E[2], r.B[0], r.B[1], r.B[2]}, n0, n1, n2};
    const SmemGather<DIM, P, G> sgather{Fs};
    unsigned my_slow = 0;
    const int D_ = D;

    // rounds of one particle per thread, the same count for every thread (the
    // bucketed deposit synchronises the CTA once per round)
    const int nrounds = (int)((p1 - p0 + blockDim.x - 1) / blockDim.x);
    bool dealt = G::BK && tile_item;  // CTA-uniform
    long long i = p0 + threadIdx.x;
    ParticleIn cur, nxt;
    cur.cell = -1;
    if (i < p1) load_particle(pb, DIM, i, r.w_const, cur);
    for (int rd = 0; rd < nrounds; ++rd, i += blockDim.x) {
        const long long inext = i + blockDim.x;
        nxt.cell = -1;
        if (inext < p1) load_particle(pb, DIM, inext, r.w_const, nxt);
        const int32_t pc = cur.cell;
        bool dep = false;  // this particle deposits in the round's bucketed deposit
        int dpk = 0;
        float dd0[3] = {0.f, 0.f, 0.f}, dd1[3] = {0.f, 0.f, 0.f}, dqw = 0.f, dqz = 0.f;
        if (pc >= 0) {
            int c[3];
            unpack_cell(r, pc, c[0], c[1], c[2]);
            bool keep = true;
            if (r.open_last) {
                int pl = c[DIM - 1] - origin;
                pl = pl < 0 ? pl + nl : pl;
                keep = pl >= r.margin && pl < nl - r.margin;  // else: left the window, absorbed
            }
            if (!keep) {
                pb.cell[i] = -1;
            } else {
                float d[3] = {cur.off[0], cur.off[1], cur.off[2]};
                float u[3] = {cur.u[0], cur.u[1], cur.u[2]};
                bool fast = tile_item;
                int rel[3] = {0, 0, 0};
                if (tile_item) {
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        int v = c[a] - org[a];
                        if (v < -D_) v += r.n[a];
                        else if (v >= G::tile(a) + D_) v -= r.n[a];
                        rel[a] = v;
                        fast = fast && v >= -D_ && v < G::tile(a) + D_;
                    }
                }
                int k[3] = {0, 0, 0};
                bool ok;
                if (fast) {
                    float d1[3] = {0.f, 0.f, 0.f}, ig;
                    ok = push_move<DIM, P>(r, sgather, rel, d, u, d1, k, ig, live);
                    if (ok) {
                        // A particle that did not move (and, in 2D, has v_z = 0)
                        // deposits exactly zero; a warp of such particles skips
                        // the deposit.
                        bool moves = DIM == 2 && u[2] != 0.f;
#pragma unroll
                        for (int a = 0; a < DIM; ++a) moves = moves || k[a] != 0 || d1[a] != d[a];
                        if (dealt) {
                            dep = moves;
                            dqw = r.q * cur.w;
                            dqz = dqw * u[2] * ig;
#pragma unroll
                            for (int a = 0; a < DIM; ++a) {
                                dpk |= ((rel[a] + 64) << (8 * a)) | ((k[a] + 1) << (24 + 2 * a));
                                dd0[a] = d[a];
                                dd1[a] = d1[a];
                            }
                        } else if (G::SPLIT && __any_sync(__activemask(), moves)) {
                            // virtual trajectories, each deposited with a no-shift window
                            const float qw = r.q * cur.w;
                            float coef[3];
#pragma unroll
                            for (int a = 0; a < DIM; ++a) coef[a] = -qw * r.d_over_dt[a];
                            const float qwvz = qw * u[2] * ig;
                            if (moves)
                                split_move<DIM, P>(rel, d, k, d1, coef, [&](const Axis<P> *ax, float frac) {
                                    if (DIM == 3) deposit3_smem<P, G>(ax, S, Jhi);
                                    else deposit2_smem<P, G>(ax, S, qwvz * frac, Jhi);
                                });
                        } else if (__any_sync(__activemask(), moves)) {
                            const float qw = r.q * cur.w;
                            Axis<P> ax[DIM];
#pragma unroll
                            for (int a = 0; a < DIM; ++a)
                                axis_window<P>(rel[a], d[a], k[a], d1[a], -qw * r.d_over_dt[a], ax[a]);
                            if (DIM == 3) deposit3_smem<P, G>(reinterpret_cast<const Axis<P> *>(ax), S, Jhi);
                            else
                                deposit2_smem<P, G>(reinterpret_cast<const Axis<P> *>(ax), S, qw * u[2] * ig, Jhi);
                        }
#pragma unroll
                        for (int a = 0; a < DIM; ++a) d[a] = d1[a];
                    }
                } else {
                    ++my_slow;
                    const SlowOut so = advance_global<DIM, P, G::SPLIT>(r, gf, c[0], c[1], c[2], d[0], d[1], d[2], u[0], u[1],
                                                              u[2], cur.w);
                    ok = so.ok != 0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        d[a] = so.d[a];
                        u[a] = so.u[a];
                        k[a] = so.k[a];
                    }
                }
                if (!ok) {  // non-finite or over-long move: drop the particle, latch the status
                    pb.cell[i] = -1;
                    atomicOr(&stp->status, kStatusBadIndex);
                } else {
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
            }
        }
        cur = nxt;
        if (dealt) {
            const int nd = deposit_round<DIM, P, G>(r, dep, dpk, dd0, dd1, dqw, dqz, S, Jhi, stg, s_cnt, s_start);
            // a tile none of whose first round's particles moved (a plasma at
            // rest in fields) deposits thread by thread from then on: no
            // barrier per round for the few particles that may move later
            if (rd == 0 && nd == 0) dealt = false;  // (nd is the same in every thread)
        }
    }
    if (my_slow) atomicAdd(&slow_cnt, my_slow);
    __syncthreads();
    if (G::TL && threadIdx.x == 0) mbar_inval(&tma_bar);  // every wait on it has returned
    if (tile_item) {
        // flush the tile's current to global J (wrapping the halo)
        const float inv = 1.f / S, inv_lo = inv * (1.f / kLoScale);
        for (int l = threadIdx.x; l < G::JVOL; l += blockDim.x) {
            int hi[3], lo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                hi[c] = Jhi[c * G::JVOL + l];
                lo[c] = Jlo[c * G::JVOL + l];
            }
            if (((hi[0] | lo[0]) | (hi[1] | lo[1]) | (hi[2] | lo[2])) == 0) continue;  // (plane padding too)
            const int lz = l / G::JPL, lxy = l - lz * G::JPL, ly = lxy / G::JX, lx = lxy - ly * G::JX;
            const int gx = modi(org[0] - G::JHX + lx, n0);
            const int gy = modi(org[1] - G::JHY + ly, n1);
            const int gz = DIM == 3 ? modi(org[2] - G::JHZ + lz, n2) : 0;
            const int g = gx + n0 * (gy + n1 * gz);
            if (r.jst == 4) {  // the node's three components in one 16-byte vector atomic
                float v[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] = fmaf((float)lo[c], inv_lo, (float)hi[c] * inv);
                atomicAdd(reinterpret_cast<float4 *>(r.J[0]) + g, make_float4(v[0], v[1], v[2], 0.f));
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (hi[c] | lo[c]) atomicAdd(r.J[c] + g, fmaf((float)lo[c], inv_lo, (float)hi[c] * inv));
            }
        }
    }
    if (threadIdx.x == 0 && slow_cnt) {
        atomicAdd(&stp->slow, (unsigned long long)slow_cnt);
        if (tile_item) atomicAdd(&stp->stray, (unsigned long long)slow_cnt);  // (not the unsorted tail)
    }
}

// ---------------------------------------------------------------- zero-field tiles
// A tile whose staged field region holds only +0 values (ahead of a laser
// front, or wherever the fields have not arrived yet) interpolates E = B = +0
// at every one of its particles.  The Boris push then returns u unchanged
// (every term adds or multiplies exact zeros; a zero momentum comes out as
// +0), so a particle at rest stays where it is and deposits no current: its
// step reads its cell (absorption at an open window's ends) and momentum and
// changes nothing else.  Such tiles are streamed by this kernel with 16-byte
// loads (four groups of four consecutive slots per thread at two CTAs of
// 256 threads per SM for tiles of 4096 slots and more, two groups at three
// CTAs per SM for smaller tiles; the ragged ends of a tile's range slot by
// slot) and no shared-memory tiles; each CTA loads its next item while it
// streams the current one.  A particle of such a tile that does
// move takes the general slow path (the gather from global memory reads the
// same zeros; the current goes to global memory by atomics) and is counted as
// a slow-path particle.  Particles outside their tile's drift region cost
// nothing here (no tile is staged) and are not counted as strays: the
// adaptive sort counts the strays that slow the staged kernel down.
constexpr int kZeroThreads = 256;
// Groups of four slots per thread and iteration: four (two CTAs per SM) for
// tiles of at least kZeroWideSlots slots, two (three CTAs per SM) for
// smaller ones, whose passes would otherwise leave threads idle.
constexpr int kZeroWideSlots = 4096;

struct ZeroCtx {
    int origin, nl;
    int last_shift;  // bit offset of the last axis in the packed cell
};

// One slot: absorption on an open last axis, the state of a particle at rest.
// Returns true when the particle moves (u != 0) and needs the slow path.
template <int DIM>
__device__ __forceinline__ bool zero_slot(const Run &r, const ZeroCtx &z, int32_t &cell, float *u)
{
    if (cell < 0) return false;
    if (r.open_last) {
        int pl = (cell >> z.last_shift) - z.origin;
        pl = pl < 0 ? pl + z.nl : pl;
        if (pl < r.margin || pl >= z.nl - r.margin) {  // left the window: absorbed
            cell = -1;
            return false;
        }
    }
    const bool rest = u[0] == 0.f && u[1] == 0.f && u[2] == 0.f;
    if (rest) u[0] = u[1] = u[2] = 0.f;  // (+0, as the push computes it)
    return !rest;
}

// The slow path for one moving particle of a zero-field tile (reloaded from
// its slot, so that no other state lives across the call).
template <int DIM, int P, bool SPLIT>
__device__ __forceinline__ void zero_mover(const Run &r, const ZeroCtx &z, const ParticleBuf &pb, long long i)
{
    RunState *stp = r.state;
    const GlobalFields gf{{r.E[0], r.E[1], r.E[2], r.B[0], r.B[1], r.B[2]}, r.n[0], r.n[1], DIM == 3 ? r.n[2] : 1};
    int c[3];
    unpack_cell(r, pb.cell[i], c[0], c[1], c[2]);
    const float w = pb.w ? pb.w[i] : r.w_const;
    const SlowOut so = advance_global<DIM, P, SPLIT>(r, gf, c[0], c[1], c[2], pb.off[0][i], pb.off[1][i],
                                              DIM == 3 ? pb.off[2][i] : 0.f, pb.u[0][i], pb.u[1][i], pb.u[2][i], w);
    if (!so.ok) {  // non-finite or over-long move: drop the particle, latch the status
        pb.cell[i] = -1;
        atomicOr(&stp->status, kStatusBadIndex);
        return;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) c[a] = wrapi(c[a] + so.k[a], r.n[a]);
    bool absorbed = false;
    if (r.open_last) {
        int pl = c[DIM - 1] - z.origin;
        pl = pl < 0 ? pl + z.nl : pl;
        absorbed = pl < r.margin || pl >= z.nl - r.margin;
    }
    pb.cell[i] = absorbed ? -1 : pack_cell(r, c[0], c[1], DIM == 3 ? c[2] : 0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) pb.off[a][i] = so.d[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) pb.u[a][i] = so.u[a];
}

template <int DIM, int P, bool SPLIT, int NG>
__global__ void __launch_bounds__(kZeroThreads, NG >= 4 ? 2 : 3) push_zero_kernel(const Run *__restrict__ runs,
                                                                                 const Item *__restrict__ list,
                                                                                 const int *__restrict__ count)
{
    __shared__ Run rs;
    const int n = *count;
    int w = blockIdx.x;
    if (w >= n) return;
    int cur = -1;
    ParticleBuf pb;
    ZeroCtx z;
    Item it = list[w];
    for (; w < n; w += gridDim.x) {
        if (it.run != cur) {  // (the same in every thread)
            __syncthreads();  // (every thread is done with the previous run's copy)
            const int *src = reinterpret_cast<const int *>(runs + it.run);
            int *dst = reinterpret_cast<int *>(&rs);
            for (int q = threadIdx.x; q < (int)(sizeof(Run) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
            cur = it.run;
            __syncthreads();
            const RunState *stp = rs.state;
            pb = rs.P[stp->buf];
            z.origin = stp->origin;
            z.nl = rs.n[DIM - 1];
            z.last_shift = DIM == 3 ? rs.bits[0] + rs.bits[1] : rs.bits[0];
        }
        const Run &r = rs;
        const int t = it.a;
        const long long p0 = r.tile_off[t], p1 = r.tile_off[t + 1];
        // (the next item is loaded while this one streams)
        if (w + (int)gridDim.x < n) it = list[w + gridDim.x];
        bool moving = false;  // this thread left a moving particle for the second pass
        // A particle at rest (u = 0) in zero fields keeps its cell, offsets
        // and momentum: the step reads its cell (absorption) and momentum
        // and writes back only what changes (an absorbed cell, a -0 momentum
        // component made +0 as the push makes it); its offsets are not
        // touched.  Four consecutive slots per thread with 16-byte accesses
        // where the arrays are 16-byte aligned; slot by slot elsewhere.
        const uintptr_t al = (uintptr_t)pb.cell | (uintptr_t)pb.u[0] | (uintptr_t)pb.u[1] | (uintptr_t)pb.u[2];
        long long v0 = (p0 + 3) & ~3ll, v1 = p1 & ~3ll;
        if ((al & 15u) != 0 || v0 >= v1) v0 = v1 = p1;
        // (NG groups of four slots per thread and iteration, all loaded
        // before any is processed: with NG = 4 a tile of 4096 slots is one
        // iteration of 256 threads, its loads all in flight together)
        const long long gend = v1 >> 2;
        for (long long g = (v0 >> 2) + threadIdx.x; g < gend; g += NG * blockDim.x) {
            long long gg[NG];
            int4 c4[NG];
            float4 u4[NG][3];
#pragma unroll
            for (int h = 0; h < NG; ++h) {
                gg[h] = g + h * (long long)blockDim.x;
                if (gg[h] >= gend) break;
                c4[h] = reinterpret_cast<const int4 *>(pb.cell)[gg[h]];
#pragma unroll
                for (int a = 0; a < 3; ++a) u4[h][a] = reinterpret_cast<const float4 *>(pb.u[a])[gg[h]];
            }
#pragma unroll
            for (int h = 0; h < NG; ++h) {
                if (gg[h] >= gend) break;
                int32_t cl[4] = {c4[h].x, c4[h].y, c4[h].z, c4[h].w};
                float uu[4][3] = {{u4[h][0].x, u4[h][1].x, u4[h][2].x}, {u4[h][0].y, u4[h][1].y, u4[h][2].y},
                                  {u4[h][0].z, u4[h][1].z, u4[h][2].z}, {u4[h][0].w, u4[h][1].w, u4[h][2].w}};
#pragma unroll
                for (int q = 0; q < 4; ++q) moving = zero_slot<DIM>(r, z, cl[q], uu[q]) || moving;
                // (a moving slot is left as it is; the second pass advances it)
                if (cl[0] != c4[h].x || cl[1] != c4[h].y || cl[2] != c4[h].z || cl[3] != c4[h].w)
                    reinterpret_cast<int4 *>(pb.cell)[gg[h]] = make_int4(cl[0], cl[1], cl[2], cl[3]);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float4 n4 = make_float4(uu[0][a], uu[1][a], uu[2][a], uu[3][a]);
                    const float4 o4 = u4[h][a];
                    if (__float_as_int(n4.x) != __float_as_int(o4.x) || __float_as_int(n4.y) != __float_as_int(o4.y) ||
                        __float_as_int(n4.z) != __float_as_int(o4.z) || __float_as_int(n4.w) != __float_as_int(o4.w))
                        reinterpret_cast<float4 *>(pb.u[a])[gg[h]] = n4;
                }
            }
        }
        // the ragged ends (and every slot when an array is not 16-byte aligned)
        const long long ends = (v0 - p0) + (p1 - v1);
        for (long long e = threadIdx.x; e < ends; e += blockDim.x) {
            const long long i = e < v0 - p0 ? p0 + e : v1 + (e - (v0 - p0));
            const int32_t c0 = pb.cell[i];
            int32_t cl = c0;
            const float u0[3] = {pb.u[0][i], pb.u[1][i], pb.u[2][i]};
            float uu[3] = {u0[0], u0[1], u0[2]};
            moving = zero_slot<DIM>(r, z, cl, uu) || moving;
            if (cl != c0) pb.cell[i] = cl;
            if (cl >= 0) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (__float_as_int(uu[a]) != __float_as_int(u0[a])) pb.u[a][i] = uu[a];
            }
        }
        // second pass, rare (a moving particle deposits, so its tile's fields
        // are soon non-zero): the tile's moving particles take the slow path,
        // reloaded one at a time so that the streaming loop above carries no
        // call (and no spilled state)
        if (__syncthreads_or(moving)) {
            unsigned slow = 0;
            for (long long i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
                if (pb.cell[i] < 0) continue;
                if (pb.u[0][i] == 0.f && pb.u[1][i] == 0.f && pb.u[2][i] == 0.f) continue;
                ++slow;
                zero_mover<DIM, P, SPLIT>(r, z, pb, i);
            }
            if (slow) atomicAdd(&r.state->slow, (unsigned long long)slow);
        }
        if (threadIdx.x == 0) atomicAdd(&r.state->streamed, (unsigned long long)(p1 - p0));
    }
}

// One CTA per item.  The persistent schedule is a kernel of its own so that
// its loop state does not compete with the item body for registers.
// live_cnt (may be null): the items past the first n_fixed are counted on
// the device; CTAs past the count return at once.
template <int DIM, int P, int TX, int TY, int TZ, int D, int V>
__global__ void __launch_bounds__(512) push_kernel(const Run *__restrict__ runs, const Item *__restrict__ items,
                                                   int tail_block, int n_fixed, const int *__restrict__ live_cnt)
{
    if (live_cnt && (int)blockIdx.x >= n_fixed + *live_cnt) return;
    process_item<DIM, P, TX, TY, TZ, D, V>(runs, items[blockIdx.x], tail_block);
}

// Persistent grid: CTAs take items from the device work queue (items
// ordered largest first) until it is empty.
template <int DIM, int P, int TX, int TY, int TZ, int D, int V>
__global__ void __launch_bounds__(512) push_queue_kernel(const Run *__restrict__ runs,
                                                         const Item *__restrict__ items, int nitems, int tail_block,
                                                         int *queue, const int *__restrict__ live_cnt)
{
    __shared__ int s_item;
    if (live_cnt) nitems += *live_cnt;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int idx = s_item;
        __syncthreads();
        if (idx >= nitems) break;
        process_item<DIM, P, TX, TY, TZ, D, V>(runs, items[idx], tail_block);
        __syncthreads();
    }
}

// nitems: items of the launch (with live_cnt: the fixed leading items; the
// device count of the others is added on the device, up to max_extra).
template <int DIM, int P, int TX, int TY, int TZ, int D, int V>
cudaError_t launch_t(const Run *runs, const Item *items, int nitems, int block, int tail_block, int *queue,
                     int persistent_ctas, cudaStream_t st, const int *live_cnt = nullptr, int max_extra = 0)
{
    using G = Geo<DIM, P, TX, TY, TZ, D, V>;
    auto k = push_kernel<DIM, P, TX, TY, TZ, D, V>;
    auto kq = push_queue_kernel<DIM, P, TX, TY, TZ, D, V>;
    static bool attr_set = false;  // raise the opt-in shared-memory limit once
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (nitems + max_extra == 0) return cudaSuccess;
    if (queue) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kq, block, G::SMEM);
        if (e != cudaSuccess) return e;
        int grid = persistent_ctas * (per_sm > 0 ? per_sm : 1);
        grid = grid < nitems + max_extra ? grid : nitems + max_extra;
        e = cudaMemsetAsync(queue, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        kq<<<grid, block, G::SMEM, st>>>(runs, items, nitems, tail_block, queue, live_cnt);
    } else {
        k<<<nitems + max_extra, block, G::SMEM, st>>>(runs, items, tail_block, nitems, live_cnt);
    }
    return cudaGetLastError();
}

template <int DIM, int P, bool SPLIT, int NG>
cudaError_t launch_zero_ng(const Run *runs, const Item *list, const int *count, int max_items, int num_sms,
                           cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_zero_kernel<DIM, P, SPLIT, NG>, kZeroThreads, 0);
    if (e != cudaSuccess) return e;
    int grid = num_sms * (per_sm > 0 ? per_sm : 1);
    grid = grid < max_items ? grid : max_items;
    push_zero_kernel<DIM, P, SPLIT, NG><<<grid, kZeroThreads, 0, st>>>(runs, list, count);
    return cudaGetLastError();
}

// wide: every run's tiles hold at least kZeroWideSlots particles
template <int DIM, int P, bool SPLIT = false>
cudaError_t launch_zero(const Run *runs, const Item *list, const int *count, int max_items, int num_sms, bool wide,
                        cudaStream_t st)
{
    if (max_items <= 0) return cudaSuccess;
    return wide ? launch_zero_ng<DIM, P, SPLIT, 4>(runs, list, count, max_items, num_sms, st)
                : launch_zero_ng<DIM, P, SPLIT, 2>(runs, list, count, max_items, num_sms, st);
}

}  // namespace push_detail
}  // namespace pic
