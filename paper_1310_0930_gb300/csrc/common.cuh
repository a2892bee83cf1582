// common.cuh -- device-side data layout of the GB300 EM-PIC timestep.
//
// A "run" is one independent simulation (grid + one particle species).  The
// plain form has one run; the batched form has many, and every phase kernel
// walks a flat list of work items that spans all runs, so one launch per
// phase covers the whole batch.
//
// Particles (Sec. 5.1): per particle a packed int32 cell index
//   cell = cx | cy << bits0 | cz << (bits0 + bits1)   (negative = dead slot)
// and FP32 offsets off[a] in [0, 1) from the cell's lower vertex, FP32
// u[3] = gamma*beta, optional FP32 weight w and optional int32 id, all in
// structure-of-arrays form, sorted by tile.  Fields are component arrays of
// n0*n1*n2 FP32 values, x fastest, without guard layers: neighbours wrap
// periodically.  An open last axis is a ring buffer whose physical origin
// (the rear of the moving window) sits at storage index `origin`.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

constexpr int kStatusOverflow = 1;  // capacity exceeded (injection / sort)
constexpr int kStatusTimeout = 2;   // a bounded wait gave up
constexpr int kStatusBadIndex = 4;  // a particle index out of range was found

struct ParticleBuf {
    int32_t *cell;
    float *off[3];
    float *u[3];
    float *w;    // nullptr: constant weight
    int32_t *id; // nullptr: not tracked
};

// Mutable per-run state, resident in device memory so that captured CUDA
// graphs replay without host-side arguments.
struct RunState {
    double time;
    long long step;
    int shifts;          // moving-window shifts so far
    int origin;          // storage index of the window's rear plane (open last axis)
    int shift_pending;   // set by the end-of-step kernel, consumed by window kernels
    int buf;             // current particle buffer (0/1)
    int status;          // latched kStatus* bits
    int pad;
    long long n_sorted;  // slots [0, n_sorted) are sorted into tiles
    long long n_total;   // slots [n_sorted, n_total) are an unsorted tail
    unsigned long long slow;       // slow-path particles of the push in progress
    unsigned long long slow_last;  // slow-path particles of the last completed step
    unsigned long long stray;      // of those, particles of tiles outside the drift region
    unsigned long long slow_acc;   // stray particle-steps since the last sort
    int since_sort;                // completed steps since the last sort
    int do_sort;                   // this step sorts (set by the sort decision)
    long long sorts;               // sorts so far
    unsigned long long streamed;   // particle slots of zero-field tiles streamed so far
    unsigned long long live_tiles; // non-empty tiles the staged kernel advanced so far
};

// Immutable per-run descriptor (device copy).
struct Run {
    int dim, order;
    int n[3];
    int bits[3];       // bit width per axis in the packed cell
    int tlog[3];       // log2 tile size per axis
    int nt[3];         // tiles per axis
    int ntiles;
    int ncell;
    float d[3], inv_d[3], dt_over_d[3], d_over_dt[3];
    float dt, qm_half_dt, q, m, w_const;
    double dt_d, d_last_d;  // exact dt and last-axis cell size for time keeping / window decisions
    double dd[3];           // exact cell sizes (laser profile positions)
    int open_last;     // 1: last axis open (Mur, absorbing), ring-buffered for the window
    int margin;        // particles kept while margin <= phys_last < n_last - margin
    int drift;         // fast-path allowance outside the tile (cells)
    float *E[3], *B[3], *J[3];
    // current layout: jst = 1: J[c] are three component arrays; jst = 4: one
    // array of float4 (x, y, z, unused) per node, J[c] = its c-th lane
    // (Sec. 5.1's four-component current), flushed by 16-byte vector atomics
    int jst;
    double *rho0;      // initial electron charge density (neutralising background), FP64 diagnostic
    float *mur;        // saved tangential E planes for Mur: [2][4][plane]
    ParticleBuf P[2];
    const void *tmap;  // 3D: six TMA tensor maps (E0..2, B0..2, 128 bytes each) for the field tile, or null
    int32_t *tile_off; // [ntiles + 1] particle offsets per tile
    int32_t *tile_cnt; // [ntiles * nsub] sort counters / cursors per (tile, sub-bucket)
    int nsub;          // sort sub-buckets per tile (power of two)
    // sub-bucket of a particle: sort_rows = 1: its row of cells along x in
    // the tile, y + ty z (y, z its cell in the tile, ty the tile's extent in
    // y; nsub = ty tz); 0: slot i % nsub
    int sort_rows;
    // per tile: 1 if some E or B value of the tile's own cells may be non-zero,
    // 0 if all are +0 (cleared by the first B half step, set by the second; set
    // for every tile whenever E or B is written from outside the timestep)
    uint8_t *fz;
    // per tile, per step (null: not kept): jt = 1 if a particle of the slow
    // path (strays, the unsorted tail, movers of zero-field tiles) deposited
    // current from a cell of the tile; quiet = 1 if the field update of the
    // tile's cells is the identity this step (no E, B or J in reach), so the
    // Yee kernels and the J reset leave them alone.  qr[a]: tiles along axis
    // a within a tile's deposit reach (drift plus the window's reach).
    uint8_t *jt, *quiet;
    int qr[3];
    long long capacity;
    // laser antenna
    int laser_on, laser_pol, laser_plane;
    double a0, omega0, waist, fwhm, t_peak;
    // moving window and injection
    int window_on;
    int ppc[3];
    double window_v, window_t0;
    double density;
    const double *knots;  // device copy of the density knots (may be nullptr)
    int n_knots;
    double z0, z1;
    // particle ids (track_ids): the loaded particles have ids 0 .. id_base-1;
    // the injection of shift k (1, 2, ...) gives its layer of `count`
    // particles the ids id_base + (k - 1) count + j
    long long id_base;
    // adjoint form armed: birth positions (lab frame, last axis) by id, which
    // the injection writes for the ids it creates (< adj_nid); else null
    float *adj_zb;
    long long adj_nid;
    RunState *state;
};

// A unit of work of a phase kernel: which run, and which part of it.
struct Item {
    int run;
    int kind;  // push: 0 = tile, 1 = tail block; yee/sort: 0 = chunk
    int a;     // tile index / chunk index
    int b;
};

__host__ __device__ inline int wrapi(int i, int n)
{
    // |i| < 2n
    i = i < 0 ? i + n : i;
    return i >= n ? i - n : i;
}

// modulo for any integer (tile staging / flush, where a halo may exceed n)
__host__ __device__ inline int modi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

__device__ inline void unpack_cell(const Run &r, int32_t c, int &cx, int &cy, int &cz)
{
    cx = c & ((1 << r.bits[0]) - 1);
    cy = (c >> r.bits[0]) & ((1 << r.bits[1]) - 1);
    cz = r.dim == 3 ? (c >> (r.bits[0] + r.bits[1])) : 0;
}

__device__ inline int32_t pack_cell(const Run &r, int cx, int cy, int cz)
{
    return cx | (cy << r.bits[0]) | (r.dim == 3 ? (cz << (r.bits[0] + r.bits[1])) : 0);
}

__device__ inline int tile_of(const Run &r, int cx, int cy, int cz)
{
    int tx = cx >> r.tlog[0], ty = cy >> r.tlog[1], tz = r.dim == 3 ? (cz >> r.tlog[2]) : 0;
    return tx + r.nt[0] * (ty + r.nt[1] * tz);
}

// physical index along the last axis (window frame) from a storage index
__device__ inline int phys_last(const Run &r, const RunState &s, int cl)
{
    if (!r.open_last) return cl;
    int nl = r.n[r.dim - 1];
    int p = cl - s.origin;
    return p < 0 ? p + nl : p;
}

// ---------------------------------------------------------------------------
// B-spline weights (Sec. 5.2 step i).  For a particle at x = c + d (cell c,
// offset d in [0,1)), node() gives the weights of the integer-located nodes
// base..base+P and half() those of the half-integer-located nodes (array
// index i meaning position i + 1/2) base..base+P.
// ---------------------------------------------------------------------------
template <int P>
struct Shape;

template <>
struct Shape<1> {
    static __device__ __forceinline__ void node(int c, float d, int &base, float *w)
    {
        base = c;
        w[0] = 1.f - d;
        w[1] = d;
    }
    static __device__ __forceinline__ void half(int c, float d, int &base, float *w)
    {
        bool hi = d >= 0.5f;
        float t = hi ? d - 0.5f : d + 0.5f;
        base = hi ? c : c - 1;
        w[0] = 1.f - t;
        w[1] = t;
    }
};

template <>
struct Shape<2> {
    static __device__ __forceinline__ void q(float t, float *w)
    {
        float a = 0.5f - t, b = 0.5f + t;
        w[0] = 0.5f * a * a;
        w[1] = 0.75f - t * t;
        w[2] = 0.5f * b * b;
    }
    static __device__ __forceinline__ void node(int c, float d, int &base, float *w)
    {
        int h = d >= 0.5f ? 1 : 0;
        base = c + h - 1;
        q(d - (float)h, w);
    }
    static __device__ __forceinline__ void half(int c, float d, int &base, float *w)
    {
        base = c - 1;
        q(d - 0.5f, w);
    }
};

template <>
struct Shape<3> {
    static __device__ __forceinline__ void cub(float f, float *w)
    {
        const float s = 1.f / 6.f;
        float g = 1.f - f, f2 = f * f, f3 = f2 * f;
        w[0] = g * g * g * s;
        w[1] = (4.f - 6.f * f2 + 3.f * f3) * s;
        w[2] = (1.f + 3.f * f + 3.f * f2 - 3.f * f3) * s;
        w[3] = f3 * s;
    }
    static __device__ __forceinline__ void node(int c, float d, int &base, float *w)
    {
        base = c - 1;
        cub(d, w);
    }
    static __device__ __forceinline__ void half(int c, float d, int &base, float *w)
    {
        bool hi = d >= 0.5f;
        base = hi ? c - 1 : c - 2;
        cub(hi ? d - 0.5f : d + 0.5f, w);
    }
};

template <>
struct Shape<4> {
    // quartic B-spline at the five nodes nearest the particle, t = position
    // minus the middle node, t in [-1/2, 1/2):
    //   |s| <= 1/2:        (115 - 120 s^2 + 48 s^4) / 192
    //   1/2 <= |s| <= 3/2: (55 + 20 |s| - 120 s^2 + 80 |s|^3 - 16 s^4) / 96
    //   3/2 <= |s| < 5/2:  (5/2 - |s|)^4 / 24
    static __device__ __forceinline__ float mid(float s)
    {
        return (55.f + s * (20.f + s * (-120.f + s * (80.f - 16.f * s)))) * (1.f / 96.f);
    }
    static __device__ __forceinline__ void q(float t, float *w)
    {
        const float a = 0.5f - t, b = 0.5f + t, t2 = t * t;
        w[0] = (a * a) * (a * a) * (1.f / 24.f);
        w[1] = mid(1.f + t);
        w[2] = (115.f + t2 * (-120.f + 48.f * t2)) * (1.f / 192.f);
        w[3] = mid(1.f - t);
        w[4] = (b * b) * (b * b) * (1.f / 24.f);
    }
    static __device__ __forceinline__ void node(int c, float d, int &base, float *w)
    {
        int h = d >= 0.5f ? 1 : 0;
        base = c + h - 2;
        q(d - (float)h, w);
    }
    static __device__ __forceinline__ void half(int c, float d, int &base, float *w)
    {
        base = c - 2;
        q(d - 0.5f, w);
    }
};

// Reach of the stencils relative to the particle's cell c, per axis:
// gather touches [c - GLO, c + GHI]; the deposit window of a move of less
// than one cell touches nodes [c - DLO, c + DHI].
template <int P>
struct Reach;
template <>
struct Reach<1> {
    static constexpr int GLO = 1, GHI = 1, DLO = 1, DHI = 2;
};
template <>
struct Reach<2> {
    static constexpr int GLO = 1, GHI = 2, DLO = 2, DHI = 3;
};
template <>
struct Reach<3> {
    static constexpr int GLO = 2, GHI = 2, DLO = 2, DHI = 3;
};
template <>
struct Reach<4> {
    static constexpr int GLO = 2, GHI = 3, DLO = 3, DHI = 4;
};

}  // namespace pic
