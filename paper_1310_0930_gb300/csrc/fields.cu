// fields.cu -- Yee FDTD update (Sec. 2; Sec. 3: a local field solver), the
// open last axis (first-order Mur fields), the laser antenna (one-way plane
// source) and the moving window (Sec. 2) on device-resident state.
//
// Per timestep: B -= (dt/2) curl E (forward differences), E += dt (curl B -
// J) (backward differences), B -= (dt/2) curl E.  Cell-parallel, one thread
// per cell and all three components, neighbours wrapped periodically.  On an
// open last axis the storage is a ring: physical index = storage - origin.
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

__device__ __forceinline__ bool laser_active(const Run &r, const RunState &s)
{
    return r.laser_on && s.shifts == 0;
}

// Incident antenna field (double precision; a few thousand values per step).
__device__ double laser_field(const Run &r, double r2, double xi)
{
    double dx = xi - r.t_peak;
    double env = exp(-2.0 * 0.69314718055994530942 * dx * dx / (r.fwhm * r.fwhm));
    return r.a0 * exp(-r2 / (r.waist * r.waist)) * env * cos(r.omega0 * dx);
}

// squared distance from the box axis of E_pol's transverse location
__device__ double laser_r2(const Run &r, int i, int j)
{
    const int last = r.dim - 1;
    double r2 = 0.0;
    int idx[2] = {i, j};
    for (int a = 0; a < last; ++a) {
        double off = (a == r.laser_pol) ? 0.5 : 0.0;
        double pos = ((double)idx[a] + off) * r.dd[a];
        double ctr = 0.5 * r.n[a] * r.dd[a];
        r2 += (pos - ctr) * (pos - ctr);
    }
    return r2;
}

// Field flags of the tiles (Run::fz): the first B half step of a timestep
// clears them (the push of the step has read them), the second sets the flag
// of every tile holding a cell whose final E or B is not +0.  The push of the
// next step streams the particles of tiles whose neighbourhood is all +0.
__device__ __forceinline__ void clear_tile_flags(const Run &r, const Seg &seg, int ri, int t)
{
    const int nthreads = (seg.start[ri + 1] - seg.start[ri]) * blockDim.x;
    for (; t < r.ntiles; t += nthreads) {
        r.fz[t] = 0;
        if (r.jt) r.jt[t] = 0;
    }
}

// The cells of a quiet tile keep E = B = J = +0 through the step (see
// quiet_kernel): their field update is the identity.
__device__ __forceinline__ bool quiet_cell(const Run &r, int i, int j, int k)
{
    return r.quiet && r.quiet[tile_of(r, i, j, k)];
}

template <int DIM>
__device__ __forceinline__ void yee_b_block(const Run *__restrict__ runs, Seg seg, int second, int vb)
{
    const int ri = seg_run(seg, vb);
    const Run &r = runs[ri];
    const int idx = (vb - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (!second && r.fz) clear_tile_flags(r, seg, ri, idx);
    if (idx >= r.ncell) return;
    const RunState &s = *r.state;
    const int n0 = r.n[0], n1 = r.n[1];
    const int i = idx % n0, j = (idx / n0) % n1, k = DIM == 3 ? idx / (n0 * n1) : 0;
    if (quiet_cell(r, i, j, k)) return;
    const int cx = (i + 1 == n0 ? 0 : i + 1) + n0 * (j + n1 * k);
    const int cy = i + n0 * ((j + 1 == n1 ? 0 : j + 1) + n1 * k);
    const float h = 0.5f * r.dt;
    const float *Ex = r.E[0], *Ey = r.E[1], *Ez = r.E[2];
    float *Bx = r.B[0], *By = r.B[1], *Bz = r.B[2];
    const float ex = Ex[idx], ey = Ey[idx], ez = Ez[idx];
    const float dEz_dy = (Ez[cy] - ez) * r.inv_d[1], dEz_dx = (Ez[cx] - ez) * r.inv_d[0];
    const float dEy_dx = (Ey[cx] - ey) * r.inv_d[0], dEx_dy = (Ex[cy] - ex) * r.inv_d[1];
    float dEy_dz = 0.f, dEx_dz = 0.f;
    if (DIM == 3) {
        const int n2 = r.n[2];
        const int cz = i + n0 * (j + n1 * (k + 1 == n2 ? 0 : k + 1));
        dEy_dz = (Ey[cz] - ey) * r.inv_d[2];
        dEx_dz = (Ex[cz] - ex) * r.inv_d[2];
    }
    const int nl = r.n[DIM - 1];
    const int il = phys_last(r, s, DIM == 3 ? k : j);
    const bool outside = r.open_last && il == nl - 1;  // half-integer positions beyond the end
    if (DIM == 3) {
        if (!outside) {
            Bx[idx] -= h * (dEz_dy - dEy_dz);
            By[idx] -= h * (dEx_dz - dEz_dx);
        }
        Bz[idx] -= h * (dEy_dx - dEx_dy);
    } else {
        if (!outside) {
            Bx[idx] -= h * dEz_dy;
            Bz[idx] -= h * (dEy_dx - dEx_dy);
        }
        By[idx] -= h * (-dEz_dx);
    }
    if (laser_active(r, s) && il == r.laser_plane - 1) {
        // B_b one plane behind saw the total E_pol: remove the incident part.
        int bcomp;
        double sgn;
        if (DIM == 3) {
            bcomp = r.laser_pol == 0 ? 1 : 0;
            sgn = r.laser_pol == 0 ? 1.0 : -1.0;
        } else {
            bcomp = 2;
            sgn = -1.0;
        }
        const double t = s.time + (second ? r.dt_d : 0.0);
        const double e = laser_field(r, laser_r2(r, i, j), t);
        r.B[bcomp][idx] += (float)(sgn * (double)h * (double)r.inv_d[DIM - 1] * e);
    }
    if (second && r.fz) {
        const unsigned nz = __float_as_uint(ex) | __float_as_uint(ey) | __float_as_uint(ez) |
                            __float_as_uint(Bx[idx]) | __float_as_uint(By[idx]) | __float_as_uint(Bz[idx]);
        if (nz) r.fz[tile_of(r, i, j, k)] = 1;  // (several threads may store the same 1)
    }
}

template <int DIM>
__global__ void yee_b_kernel(const Run *__restrict__ runs, Seg seg, int second)
{
    for (int vb = blockIdx.x; vb < seg.nblocks; vb += gridDim.x) yee_b_block<DIM>(runs, seg, second, vb);
}

template <int DIM>
__device__ __forceinline__ void yee_e_block(const Run *__restrict__ runs, Seg seg, int vb)
{
    const int ri = seg_run(seg, vb);
    const Run &r = runs[ri];
    const int idx = (vb - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (idx >= r.ncell) return;
    const RunState &s = *r.state;
    const int n0 = r.n[0], n1 = r.n[1];
    const int i = idx % n0, j = (idx / n0) % n1, k = DIM == 3 ? idx / (n0 * n1) : 0;
    if (quiet_cell(r, i, j, k)) return;
    const int mx = (i == 0 ? n0 - 1 : i - 1) + n0 * (j + n1 * k);
    const int my = i + n0 * ((j == 0 ? n1 - 1 : j - 1) + n1 * k);
    const float dt = r.dt;
    float *Ex = r.E[0], *Ey = r.E[1], *Ez = r.E[2];
    const float *Bx = r.B[0], *By = r.B[1], *Bz = r.B[2];
    const float bx = Bx[idx], by = By[idx], bz = Bz[idx];
    const float dBz_dy = (bz - Bz[my]) * r.inv_d[1], dBz_dx = (bz - Bz[mx]) * r.inv_d[0];
    const float dBy_dx = (by - By[mx]) * r.inv_d[0], dBx_dy = (bx - Bx[my]) * r.inv_d[1];
    float dBy_dz = 0.f, dBx_dz = 0.f;
    if (DIM == 3) {
        const int n2 = r.n[2];
        const int mz = i + n0 * (j + n1 * (k == 0 ? n2 - 1 : k - 1));
        dBy_dz = (by - By[mz]) * r.inv_d[2];
        dBx_dz = (bx - Bx[mz]) * r.inv_d[2];
    }
    float nv[3];
    const long long ji = (long long)idx * r.jst;
    nv[0] = Ex[idx] + dt * (dBz_dy - dBy_dz - r.J[0][ji]);
    nv[1] = Ey[idx] + dt * (dBx_dz - dBz_dx - r.J[1][ji]);
    nv[2] = Ez[idx] + dt * (dBy_dx - dBx_dy - r.J[2][ji]);
    const int nl = r.n[DIM - 1];
    const int il = phys_last(r, s, DIM == 3 ? k : j);
    if (r.open_last) {
        const int t0 = 0, t1 = DIM == 3 ? 1 : 2, nrm = DIM == 3 ? 2 : 1;
        if (il == 0 || il == nl - 1) {  // tangential: set by the Mur update afterwards
            nv[t0] = Ex[idx];
            nv[t1] = t1 == 1 ? Ey[idx] : Ez[idx];
        }
        if (il == nl - 1) nv[nrm] = 0.f;
    }
    if (laser_active(r, s) && il == r.laser_plane) {
        // E_pol on the plane saw the scattered B_b one plane behind: add the incident B.
        const double th = s.time + 0.5 * r.dt_d;
        const double e = laser_field(r, laser_r2(r, i, j), th + 0.5 * r.d_last_d);
        nv[r.laser_pol] += (float)((double)dt * (double)r.inv_d[DIM - 1] * e);
    }
    Ex[idx] = nv[0];
    Ey[idx] = nv[1];
    Ez[idx] = nv[2];
}

template <int DIM>
__global__ void yee_e_kernel(const Run *__restrict__ runs, Seg seg)
{
    for (int vb = blockIdx.x; vb < seg.nblocks; vb += gridDim.x) yee_e_block<DIM>(runs, seg, vb);
}

// ---------------------------------------------------------------------------
// The same updates with four consecutive x cells per thread: rows of n0 % 4 ==
// 0 cells, 16-byte vector loads and stores of the own cells and of the +-y,
// +-z neighbour rows, one scalar load for the x neighbour across the quad.
// Launched on the cell segments with kQuadThreads threads per block (each
// block then covers the kBlock cells of one cell-segment block).
// ---------------------------------------------------------------------------
constexpr int kQuadThreads = kBlock / 4;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) { *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ void unpack4(const float4 q, float (&v)[4])
{
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}

// The four cells idx0 .. idx0+3 (one x row, one tile) of a B half step.
template <int DIM>
__device__ __forceinline__ void yee_b_quad_group(const Run &r, int second, int idx0)
{
    const RunState &s = *r.state;
    const int n0 = r.n[0], n1 = r.n[1];
    const int i0 = idx0 % n0, row = idx0 / n0, j = row % n1, k = DIM == 3 ? row / n1 : 0;
    const int xn = i0 + 4 == n0 ? idx0 + 4 - n0 : idx0 + 4;  // x neighbour of the last cell
    const int cy = i0 + n0 * ((j + 1 == n1 ? 0 : j + 1) + n1 * k);
    const float h = 0.5f * r.dt;
    float ex[5], ey[5], ez[5], exy[4], ezy[4], exz[4] = {0, 0, 0, 0}, eyz[4] = {0, 0, 0, 0};
    float bx[4], by[4], bz[4];
    {
        float t[4];
        unpack4(ld4(r.E[0] + idx0), t);
        for (int e = 0; e < 4; ++e) ex[e] = t[e];
        unpack4(ld4(r.E[1] + idx0), t);
        for (int e = 0; e < 4; ++e) ey[e] = t[e];
        unpack4(ld4(r.E[2] + idx0), t);
        for (int e = 0; e < 4; ++e) ez[e] = t[e];
    }
    ey[4] = r.E[1][xn];
    ez[4] = r.E[2][xn];
    unpack4(ld4(r.E[0] + cy), exy);
    unpack4(ld4(r.E[2] + cy), ezy);
    if (DIM == 3) {
        const int n2 = r.n[2];
        const int cz = i0 + n0 * (j + n1 * (k + 1 == n2 ? 0 : k + 1));
        unpack4(ld4(r.E[0] + cz), exz);
        unpack4(ld4(r.E[1] + cz), eyz);
    }
    unpack4(ld4(r.B[0] + idx0), bx);
    unpack4(ld4(r.B[1] + idx0), by);
    unpack4(ld4(r.B[2] + idx0), bz);
    const int nl = r.n[DIM - 1];
    const int il = phys_last(r, s, DIM == 3 ? k : j);
    const bool outside = r.open_last && il == nl - 1;  // half-integer positions beyond the end
    const bool laser = laser_active(r, s) && il == r.laser_plane - 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float dEz_dy = (ezy[e] - ez[e]) * r.inv_d[1], dEz_dx = (ez[e + 1] - ez[e]) * r.inv_d[0];
        const float dEy_dx = (ey[e + 1] - ey[e]) * r.inv_d[0], dEx_dy = (exy[e] - ex[e]) * r.inv_d[1];
        float dEy_dz = 0.f, dEx_dz = 0.f;
        if (DIM == 3) {
            dEy_dz = (eyz[e] - ey[e]) * r.inv_d[2];
            dEx_dz = (exz[e] - ex[e]) * r.inv_d[2];
        }
        if (DIM == 3) {
            if (!outside) {
                bx[e] -= h * (dEz_dy - dEy_dz);
                by[e] -= h * (dEx_dz - dEz_dx);
            }
            bz[e] -= h * (dEy_dx - dEx_dy);
        } else {
            if (!outside) {
                bx[e] -= h * dEz_dy;
                bz[e] -= h * (dEy_dx - dEx_dy);
            }
            by[e] -= h * (-dEz_dx);
        }
        if (laser) {  // B_b one plane behind saw the total E_pol: remove the incident part
            const double t = s.time + (second ? r.dt_d : 0.0);
            const double f = laser_field(r, laser_r2(r, i0 + e, j), t);
            const float add = (float)((DIM == 3 ? (r.laser_pol == 0 ? 1.0 : -1.0) : -1.0) * (double)h *
                                      (double)r.inv_d[DIM - 1] * f);
            if (DIM == 3) {
                if (r.laser_pol == 0) by[e] += add;
                else bx[e] += add;
            } else {
                bz[e] += add;
            }
        }
    }
    st4(r.B[0] + idx0, bx);
    st4(r.B[1] + idx0, by);
    st4(r.B[2] + idx0, bz);
    if (second && r.fz) {
        unsigned nz = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            nz |= __float_as_uint(ex[e]) | __float_as_uint(ey[e]) | __float_as_uint(ez[e]) | __float_as_uint(bx[e]) |
                  __float_as_uint(by[e]) | __float_as_uint(bz[e]);
        // (tiles are at least 4 cells wide along x and rows start on multiples
        // of 4, so the four cells share one tile; several threads may store the same 1)
        if (nz) r.fz[tile_of(r, i0, j, k)] = 1;
    }
}

template <int DIM>
__global__ void yee_b_quad_kernel(const Run *__restrict__ runs, Seg seg, int second)
{
    for (int vb = blockIdx.x; vb < seg.nblocks; vb += gridDim.x) {
        const int ri = seg_run(seg, vb);
        const Run &r = runs[ri];
        const int idx0 = (vb - seg.start[ri]) * kBlock + 4 * threadIdx.x;
        if (!second && r.fz) clear_tile_flags(r, seg, ri, (vb - seg.start[ri]) * blockDim.x + threadIdx.x);
        if (idx0 < r.ncell) yee_b_quad_group<DIM>(r, second, idx0);
    }
}

// The four cells idx0 .. idx0+3 (one x row, one tile) of the E step.
template <int DIM>
__device__ __forceinline__ void yee_e_quad_group(const Run &r, int idx0)
{
    const RunState &s = *r.state;
    const int n0 = r.n[0], n1 = r.n[1];
    const int i0 = idx0 % n0, row = idx0 / n0, j = row % n1, k = DIM == 3 ? row / n1 : 0;
    const int xm = i0 == 0 ? idx0 + n0 - 1 : idx0 - 1;  // x neighbour of the first cell
    const int my = i0 + n0 * ((j == 0 ? n1 - 1 : j - 1) + n1 * k);
    const float dt = r.dt;
    // b?[0] is the -x neighbour of cell 0, b?[1 + e] cell e
    float bx[4], by[5], bz[5], bxy[4], bzy[4], bxz[4] = {0, 0, 0, 0}, byz[4] = {0, 0, 0, 0};
    float ex[4], ey[4], ez[4], jx[4], jy[4], jz[4];
    {
        float t[4];
        unpack4(ld4(r.B[0] + idx0), bx);
        unpack4(ld4(r.B[1] + idx0), t);
        for (int e = 0; e < 4; ++e) by[e + 1] = t[e];
        unpack4(ld4(r.B[2] + idx0), t);
        for (int e = 0; e < 4; ++e) bz[e + 1] = t[e];
    }
    by[0] = r.B[1][xm];
    bz[0] = r.B[2][xm];
    unpack4(ld4(r.B[0] + my), bxy);
    unpack4(ld4(r.B[2] + my), bzy);
    if (DIM == 3) {
        const int n2 = r.n[2];
        const int mz = i0 + n0 * (j + n1 * (k == 0 ? n2 - 1 : k - 1));
        unpack4(ld4(r.B[0] + mz), bxz);
        unpack4(ld4(r.B[1] + mz), byz);
    }
    unpack4(ld4(r.E[0] + idx0), ex);
    unpack4(ld4(r.E[1] + idx0), ey);
    unpack4(ld4(r.E[2] + idx0), ez);
    if (r.jst == 4) {  // four-component nodes: one 16-byte load per cell
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 q = ld4(r.J[0] + 4ll * (idx0 + e));
            jx[e] = q.x;
            jy[e] = q.y;
            jz[e] = q.z;
        }
    } else {
        unpack4(ld4(r.J[0] + idx0), jx);
        unpack4(ld4(r.J[1] + idx0), jy);
        unpack4(ld4(r.J[2] + idx0), jz);
    }
    const int nl = r.n[DIM - 1];
    const int il = phys_last(r, s, DIM == 3 ? k : j);
    const bool tang = r.open_last && (il == 0 || il == nl - 1);  // tangential: set by the Mur update
    const bool norm0 = r.open_last && il == nl - 1;
    const bool laser = laser_active(r, s) && il == r.laser_plane;
    float nx[4], ny[4], nz[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float dBz_dy = (bz[e + 1] - bzy[e]) * r.inv_d[1], dBz_dx = (bz[e + 1] - bz[e]) * r.inv_d[0];
        const float dBy_dx = (by[e + 1] - by[e]) * r.inv_d[0], dBx_dy = (bx[e] - bxy[e]) * r.inv_d[1];
        float dBy_dz = 0.f, dBx_dz = 0.f;
        if (DIM == 3) {
            dBy_dz = (by[e + 1] - byz[e]) * r.inv_d[2];
            dBx_dz = (bx[e] - bxz[e]) * r.inv_d[2];
        }
        float nv[3];
        nv[0] = ex[e] + dt * (dBz_dy - dBy_dz - jx[e]);
        nv[1] = ey[e] + dt * (dBx_dz - dBz_dx - jy[e]);
        nv[2] = ez[e] + dt * (dBy_dx - dBx_dy - jz[e]);
        if (tang) {
            nv[0] = ex[e];
            if (DIM == 3) nv[1] = ey[e];
            else nv[2] = ez[e];
        }
        if (norm0) nv[DIM == 3 ? 2 : 1] = 0.f;
        if (laser) {  // E_pol on the plane saw the scattered B_b one plane behind: add the incident B
            const double th = s.time + 0.5 * r.dt_d;
            const double f = laser_field(r, laser_r2(r, i0 + e, j), th + 0.5 * r.d_last_d);
            nv[r.laser_pol] += (float)((double)dt * (double)r.inv_d[DIM - 1] * f);
        }
        nx[e] = nv[0];
        ny[e] = nv[1];
        nz[e] = nv[2];
    }
    st4(r.E[0] + idx0, nx);
    st4(r.E[1] + idx0, ny);
    st4(r.E[2] + idx0, nz);
}

template <int DIM>
__global__ void yee_e_quad_kernel(const Run *__restrict__ runs, Seg seg)
{
    for (int vb = blockIdx.x; vb < seg.nblocks; vb += gridDim.x) {
        const int ri = seg_run(seg, vb);
        const Run &r = runs[ri];
        const int idx0 = (vb - seg.start[ri]) * kBlock + 4 * threadIdx.x;
        if (idx0 < r.ncell) yee_e_quad_group<DIM>(r, idx0);
    }
}

// The same over a list of rows of tiles along x (those with a tile that is
// not quiet this step): one row of tiles per block iteration, its cells in
// x rows of four-cell groups (whole rows: the access pattern of the cell
// grid).  Entry a of a row is ty + nt[1] tz.
__device__ __forceinline__ int tile_group_cell(const Run &r, int a, int g, int &valid)
{
    const int G0 = r.n[0] >> 2, T1 = 1 << r.tlog[1];
    const int gx = g % G0, gy = (g / G0) % T1, gz = g / (G0 * T1);
    const int ty = a % r.nt[1], tz = a / r.nt[1];
    const int y = (ty << r.tlog[1]) + gy, z = r.dim == 3 ? (tz << r.tlog[2]) + gz : 0;
    valid = y < r.n[1] && (r.dim != 3 || z < r.n[2]);
    return 4 * gx + r.n[0] * (y + r.n[1] * z);
}

__device__ __forceinline__ int tile_groups(const Run &r)
{
    return (r.n[0] >> 2) * (1 << r.tlog[1]) * (r.dim == 3 ? 1 << r.tlog[2] : 1);
}

template <int DIM>
__global__ void yee_b_list_kernel(const Run *__restrict__ runs, const Item *__restrict__ list,
                                  const int *__restrict__ count, int second)
{
    const int n = *count;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const Item it = list[e];
        const Run &r = runs[it.run];
        const int ng = tile_groups(r);
        for (int g = threadIdx.x; g < ng; g += blockDim.x) {
            int valid;
            const int idx0 = tile_group_cell(r, it.a, g, valid);
            if (valid) yee_b_quad_group<DIM>(r, second, idx0);
        }
    }
}

template <int DIM>
__global__ void yee_e_list_kernel(const Run *__restrict__ runs, const Item *__restrict__ list,
                                  const int *__restrict__ count)
{
    const int n = *count;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const Item it = list[e];
        const Run &r = runs[it.run];
        const int ng = tile_groups(r);
        for (int g = threadIdx.x; g < ng; g += blockDim.x) {
            int valid;
            const int idx0 = tile_group_cell(r, it.a, g, valid);
            if (valid) yee_e_quad_group<DIM>(r, idx0);
        }
    }
}

// J reset of the tiles a list holds (four cells per thread, 16-byte stores)
__global__ void zero_j_list_kernel(const Run *__restrict__ runs, const Item *__restrict__ list,
                                   const int *__restrict__ count)
{
    const int n = *count;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const Item it = list[e];
        const Run &r = runs[it.run];
        const int ng = tile_groups(r);
        for (int g = threadIdx.x; g < ng; g += blockDim.x) {
            int valid;
            const int idx0 = tile_group_cell(r, it.a, g, valid);
            if (!valid) continue;
            if (r.jst == 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) reinterpret_cast<float4 *>(r.J[0])[idx0 + q] = z;
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) *reinterpret_cast<float4 *>(r.J[c] + idx0) = z;
            }
        }
    }
}

// Tile flags of the step that just ended: cleared once the quiet tiles are
// known (the B half steps set the field flags again, the slow path the
// deposit flags).
__global__ void clear_flags_kernel(const Run *__restrict__ runs)
{
    const Run &r = runs[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r.ntiles) return;
    r.fz[t] = 0;
    if (r.jt) r.jt[t] = 0;
}

__device__ __forceinline__ void zero_j_block(const Run *__restrict__ runs, Seg seg, int vb)
{
    const int ri = seg_run(seg, vb);
    const Run &r = runs[ri];
    const int idx = (vb - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (idx >= r.ncell) return;
    if (r.quiet) {  // a tile quiet at the last step kept J = 0 (no deposit reached it)
        const int n0 = r.n[0], n1 = r.n[1], row = idx / n0;
        if (quiet_cell(r, idx % n0, row % n1, r.dim == 3 ? row / n1 : 0)) return;
    }
    if (r.jst == 4) {
        reinterpret_cast<float4 *>(r.J[0])[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    r.J[0][idx] = 0.f;
    r.J[1][idx] = 0.f;
    r.J[2][idx] = 0.f;
}

__global__ void zero_j_kernel(const Run *__restrict__ runs, Seg seg)
{
    for (int vb = blockIdx.x; vb < seg.nblocks; vb += gridDim.x) zero_j_block(runs, seg, vb);
}

// Four cells per thread (kQuadThreads per block of kBlock cells), 16-byte stores.
__device__ __forceinline__ void zero_j_quad_block(const Run *__restrict__ runs, Seg seg, int vb)
{
    const int ri = seg_run(seg, vb);
    const Run &r = runs[ri];
    const int idx0 = (vb - seg.start[ri]) * kBlock + 4 * threadIdx.x;
    if (idx0 >= r.ncell) return;
    if (r.quiet) {  // a tile quiet at the last step kept J = 0 (the four cells share one tile)
        const int n0 = r.n[0], n1 = r.n[1], row = idx0 / n0;
        if (quiet_cell(r, idx0 % n0, row % n1, r.dim == 3 ? row / n1 : 0)) return;
    }
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r.jst == 4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) reinterpret_cast<float4 *>(r.J[0])[idx0 + e] = z;
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<float4 *>(r.J[c] + idx0) = z;
}

__global__ void zero_j_quad_kernel(const Run *__restrict__ runs, Seg seg)
{
    for (int vb = blockIdx.x; vb < seg.nblocks; vb += gridDim.x) zero_j_quad_block(runs, seg, vb);
}

// Grid of the cell kernels: a few resident blocks per SM that walk the cell
// segment's blocks (most blocks of a quiet box return at once; launching
// one block per 256 cells would cost more than their work).
int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 1;
    }
    return sms;
}

int cell_grid(const Seg &cells, int blocks_per_sm)
{
    const int g = num_sms() * blocks_per_sm;
    return cells.nblocks < g ? (cells.nblocks > 0 ? cells.nblocks : 1) : g;
}

// Quiet tiles of this step, computed after the particle phase and before the
// field update: a tile is quiet when no tile within twice its deposit reach
// (2 qr tiles per axis) has a field flag set (E and B were +0 there after the
// last step: no live tile's particles can have deposited into this tile, and
// no field can propagate into it within the step's three half updates, at
// most one cell each), no slow-path particle within its reach (qr) deposited
// this step, and the antenna's plane is not within its reach.  Such a tile's
// E, B and J are +0 before the update and stay +0 after it.
__global__ void quiet_kernel(const Run *__restrict__ runs)
{
    const Run &r = runs[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!r.quiet || t >= r.ntiles) return;
    const int d3 = r.dim == 3;
    const int nt0 = r.nt[0], nt1 = r.nt[1], nt2 = d3 ? r.nt[2] : 1;
    const int tx = t % nt0, ty = (t / nt0) % nt1, tz = d3 ? t / (nt0 * nt1) : 0;
    const int q0 = r.qr[0], q1 = r.qr[1], q2 = d3 ? r.qr[2] : 0;
    bool q = true;
    for (int dz = -2 * q2; dz <= 2 * q2 && q; ++dz) {
        const int z = modi(tz + dz, nt2);
        for (int dy = -2 * q1; dy <= 2 * q1 && q; ++dy) {
            const int y = modi(ty + dy, nt1);
            for (int dx = -2 * q0; dx <= 2 * q0 && q; ++dx) {
                const int u = modi(tx + dx, nt0) + nt0 * (y + nt1 * z);
                const bool near = abs(dx) <= q0 && abs(dy) <= q1 && abs(dz) <= q2;
                q = !r.fz[u] && !(near && r.jt[u]);
            }
        }
    }
    if (q && r.laser_on) {  // the antenna's plane (storage index) within reach
        const int nl = r.n[r.dim - 1], ntl = d3 ? nt2 : nt1, ql = d3 ? q2 : q1;
        int st = r.laser_plane + r.state->origin;
        st = st >= nl ? st - nl : st;
        int dl = abs((d3 ? tz : ty) - (st >> r.tlog[r.dim - 1]));
        dl = dl < ntl - dl ? dl : ntl - dl;
        q = dl > ql;
    }
    r.quiet[t] = q ? 1 : 0;
}

// The rows of tiles along x with a tile that is not quiet, for the field
// update (one thread per row, warp-aggregated appends).
__global__ void quiet_rows_kernel(const Run *__restrict__ runs, Item *__restrict__ nq, int *__restrict__ nq_count)
{
    const Run &r = runs[blockIdx.y];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int nrows = r.nt[1] * (r.dim == 3 ? r.nt[2] : 1);
    bool busy = false;
    if (r.quiet && a < nrows)
        for (int tx = 0; tx < r.nt[0] && !busy; ++tx) busy = !r.quiet[tx + r.nt[0] * a];
    const unsigned m = __ballot_sync(0xffffffffu, busy);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(nq_count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (busy) nq[base + __popc(m & ((1u << lane) - 1u))] = Item{(int)blockIdx.y, 0, a, 0};
}

// storage offset of physical plane `pl` (last axis) and transverse position q
__device__ __forceinline__ int plane_index(const Run &r, const RunState &s, int pl, int q)
{
    const int nl = r.n[r.dim - 1];
    const int plane = r.ncell / nl;
    int st = pl + s.origin;
    st = st >= nl ? st - nl : st;
    return q + plane * st;
}

// Mur: keep E^n of the two tangential components on physical planes 0, 1,
// nl-2, nl-1 before the E update.
__global__ void mur_save_kernel(const Run *__restrict__ runs, Seg seg)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    if (!r.open_last) return;
    const int nl = r.n[r.dim - 1];
    const int plane = r.ncell / nl;
    const int q = (blockIdx.x - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (q >= plane) return;
    const RunState &s = *r.state;
    const int pls[4] = {0, 1, nl - 2, nl - 1};
    const float *F[2] = {r.E[0], r.dim == 3 ? r.E[1] : r.E[2]};
    for (int t = 0; t < 2; ++t)
        for (int p = 0; p < 4; ++p) r.mur[(t * 4 + p) * plane + q] = F[t][plane_index(r, s, pls[p], q)];
}

// first-order Mur at normal incidence:
// F_0^{n+1} = F_1^n + (dt - d)/(dt + d) (F_1^{n+1} - F_0^n), likewise at the far end.
__global__ void mur_apply_kernel(const Run *__restrict__ runs, Seg seg)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    if (!r.open_last) return;
    const int nl = r.n[r.dim - 1];
    const int plane = r.ncell / nl;
    const int q = (blockIdx.x - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (q >= plane) return;
    const RunState &s = *r.state;
    const float dl = r.d[r.dim - 1];
    const float coef = (r.dt - dl) / (r.dt + dl);
    float *F[2] = {r.E[0], r.dim == 3 ? r.E[1] : r.E[2]};
    for (int t = 0; t < 2; ++t) {
        const float o0 = r.mur[(t * 4 + 0) * plane + q], o1 = r.mur[(t * 4 + 1) * plane + q];
        const float om1 = r.mur[(t * 4 + 2) * plane + q], om = r.mur[(t * 4 + 3) * plane + q];
        const int c0 = plane_index(r, s, 0, q), c1 = plane_index(r, s, 1, q);
        const int cm = plane_index(r, s, nl - 1, q), cm1 = plane_index(r, s, nl - 2, q);
        F[t][c0] = o1 + coef * (F[t][c1] - o0);
        F[t][cm] = om1 + coef * (F[t][cm1] - om);
    }
}

// time advance and the moving-window decision (one thread per run)
__global__ void end_step_kernel(const Run *__restrict__ runs, int nruns)
{
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    RunState &s = *r.state;
    s.time += r.dt_d;
    s.step += 1;
    s.slow_last = s.slow;
    s.slow_acc += s.stray;  // (the unsorted tail is bounded by the longest interval)
    s.stray = 0;
    s.since_sort += 1;
    s.slow = 0;
    s.shift_pending = 0;
    if (r.window_on && s.time >= r.window_t0) {
        const double travelled = r.window_v * (s.time - r.window_t0);
        if (travelled >= (double)(s.shifts + 1) * r.d_last_d) {
            const int nl = r.n[r.dim - 1];
            s.shifts += 1;
            s.origin = s.origin + 1 == nl ? 0 : s.origin + 1;
            s.shift_pending = 1;
        }
    }
}

// zero E and B on the plane that became the new front (storage origin-1)
__global__ void window_zero_kernel(const Run *__restrict__ runs, Seg seg)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    const RunState &s = *r.state;
    if (!s.shift_pending) return;
    const int nl = r.n[r.dim - 1];
    const int plane = r.ncell / nl;
    const int q = (blockIdx.x - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (q >= plane) return;
    const int idx = plane_index(r, s, nl - 1, q);
    for (int c = 0; c < 3; ++c) {
        r.E[c][idx] = 0.f;
        r.B[c][idx] = 0.f;
    }
}

__device__ double profile_density(const Run &r, double z)
{
    if (r.n_knots <= 0 || r.knots == nullptr) return r.density;
    if (r.n_knots == 1) return r.knots[0];
    double f = (z - r.z0) / (r.z1 - r.z0) * (r.n_knots - 1);
    if (f <= 0.0) return r.knots[0];
    if (f >= r.n_knots - 1) return r.knots[r.n_knots - 1];
    int i = (int)floor(f);
    double t = f - i;
    return r.knots[i] * (1.0 - t) + r.knots[i + 1] * t;
}

// Inject one cold, regularly placed layer of cells at physical last-axis
// index nl - margin - 1 (appended to the unsorted tail, slot n_total + j for
// the j-th particle of the layer).
__global__ void window_inject_kernel(const Run *__restrict__ runs, Seg seg)
{
    const int ri = seg_run(seg, blockIdx.x);
    const Run &r = runs[ri];
    const RunState &s = *r.state;
    if (!s.shift_pending) return;
    const int dim = r.dim, nl = r.n[dim - 1];
    const int ncol = r.ncell / nl;
    const int ppc_t = r.ppc[0] * r.ppc[1] * (dim == 3 ? r.ppc[2] : 1);
    const long long count = (long long)ncol * ppc_t;
    const long long q = (long long)(blockIdx.x - seg.start[ri]) * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const long long base = s.n_total;
    if (base + count > r.capacity) return;  // overflow is latched by the commit kernel
    const int col = (int)(q / ppc_t);
    int sub = (int)(q % ppc_t);
    int m[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        m[a] = sub % r.ppc[a];
        sub /= r.ppc[a];
    }
    int c[3] = {0, 0, 0};
    c[0] = col % r.n[0];
    if (dim == 3) c[1] = col / r.n[0];
    const int kcell = nl - r.margin - 1;
    int st = kcell + s.origin;
    c[dim - 1] = st >= nl ? st - nl : st;
    const ParticleBuf pb = r.P[s.buf];
    const long long slot = base + q;
    pb.cell[slot] = pack_cell(r, c[0], c[1], dim == 3 ? c[2] : 0);
    float off_last = 0.f;
    for (int a = 0; a < dim; ++a) {
        float o = ((float)m[a] + 0.5f) / (float)r.ppc[a];
        pb.off[a][slot] = o;
        if (a == dim - 1) off_last = o;
    }
    pb.u[0][slot] = 0.f;
    pb.u[1][slot] = 0.f;
    pb.u[2][slot] = 0.f;
    const double zlab = ((double)kcell + (double)off_last + (double)s.shifts) * r.d_last_d;
    if (pb.w) pb.w[slot] = (float)(profile_density(r, zlab) / ppc_t);
    if (pb.id) {
        const long long id = r.id_base + (long long)(s.shifts - 1) * count + q;
        pb.id[slot] = id < 2147483647ll ? (int32_t)id : -1;
        if (r.adj_zb && id < r.adj_nid) r.adj_zb[id] = (float)zlab;
    }
}

__global__ void window_commit_kernel(const Run *__restrict__ runs, int nruns)
{
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= nruns) return;
    const Run &r = runs[ri];
    RunState &s = *r.state;
    if (!s.shift_pending) return;
    const int nl = r.n[r.dim - 1];
    const long long count =
        (long long)(r.ncell / nl) * r.ppc[0] * r.ppc[1] * (r.dim == 3 ? r.ppc[2] : 1);
    if (s.n_total + count > r.capacity) s.status |= kStatusOverflow;
    else s.n_total += count;
    s.shift_pending = 0;
}

}  // namespace

cudaError_t launch_zero_j(const Run *runs, Seg cells, bool quad, cudaStream_t st)
{
    if (quad) zero_j_quad_kernel<<<cell_grid(cells, 24), kQuadThreads, 0, st>>>(runs, cells);
    else zero_j_kernel<<<cell_grid(cells, 8), kBlock, 0, st>>>(runs, cells);
    return cudaGetLastError();
}

cudaError_t launch_yee_b(int dim, const Run *runs, Seg cells, int second_half, bool quad, cudaStream_t st)
{
    if (quad) {
        const int g = cell_grid(cells, 24);
        if (dim == 3) yee_b_quad_kernel<3><<<g, kQuadThreads, 0, st>>>(runs, cells, second_half);
        else yee_b_quad_kernel<2><<<g, kQuadThreads, 0, st>>>(runs, cells, second_half);
    } else {
        const int g = cell_grid(cells, 8);
        if (dim == 3) yee_b_kernel<3><<<g, kBlock, 0, st>>>(runs, cells, second_half);
        else yee_b_kernel<2><<<g, kBlock, 0, st>>>(runs, cells, second_half);
    }
    return cudaGetLastError();
}

cudaError_t launch_yee_e(int dim, const Run *runs, Seg cells, bool quad, cudaStream_t st)
{
    if (quad) {
        const int g = cell_grid(cells, 24);
        if (dim == 3) yee_e_quad_kernel<3><<<g, kQuadThreads, 0, st>>>(runs, cells);
        else yee_e_quad_kernel<2><<<g, kQuadThreads, 0, st>>>(runs, cells);
    } else {
        const int g = cell_grid(cells, 8);
        if (dim == 3) yee_e_kernel<3><<<g, kBlock, 0, st>>>(runs, cells);
        else yee_e_kernel<2><<<g, kBlock, 0, st>>>(runs, cells);
    }
    return cudaGetLastError();
}

cudaError_t launch_mur_save(const Run *runs, Seg planes, cudaStream_t st)
{
    mur_save_kernel<<<planes.nblocks, kBlock, 0, st>>>(runs, planes);
    return cudaGetLastError();
}

cudaError_t launch_mur_apply(const Run *runs, Seg planes, cudaStream_t st)
{
    mur_apply_kernel<<<planes.nblocks, kBlock, 0, st>>>(runs, planes);
    return cudaGetLastError();
}

cudaError_t launch_quiet(const Run *runs, int nruns, int max_tiles, Item *nq, int *nq_count, cudaStream_t st)
{
    if (max_tiles <= 0) return cudaSuccess;
    const dim3 g((max_tiles + kBlock - 1) / kBlock, nruns);
    quiet_kernel<<<g, kBlock, 0, st>>>(runs);
    quiet_rows_kernel<<<g, kBlock, 0, st>>>(runs, nq, nq_count);  // (rows <= tiles)
    clear_flags_kernel<<<g, kBlock, 0, st>>>(runs);
    return cudaGetLastError();
}

cudaError_t launch_field_list(int which, int dim, const Run *runs, const Item *nq, const int *nq_count, int second,
                              cudaStream_t st)
{
    const int g = num_sms() * 4;  // (resident blocks walk the list)
    constexpr int kListThreads = 256;
    if (which == 0) zero_j_list_kernel<<<g, kListThreads, 0, st>>>(runs, nq, nq_count);
    else if (which == 1) {
        if (dim == 3) yee_b_list_kernel<3><<<g, kListThreads, 0, st>>>(runs, nq, nq_count, second);
        else yee_b_list_kernel<2><<<g, kListThreads, 0, st>>>(runs, nq, nq_count, second);
    } else {
        if (dim == 3) yee_e_list_kernel<3><<<g, kListThreads, 0, st>>>(runs, nq, nq_count);
        else yee_e_list_kernel<2><<<g, kListThreads, 0, st>>>(runs, nq, nq_count);
    }
    return cudaGetLastError();
}

cudaError_t launch_end_step(const Run *runs, int nruns, cudaStream_t st)
{
    end_step_kernel<<<(nruns + 127) / 128, 128, 0, st>>>(runs, nruns);
    return cudaGetLastError();
}

cudaError_t launch_window(const Run *runs, Seg planes, Seg inject, cudaStream_t st)
{
    window_zero_kernel<<<planes.nblocks, kBlock, 0, st>>>(runs, planes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    window_inject_kernel<<<inject.nblocks, kBlock, 0, st>>>(runs, inject);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    window_commit_kernel<<<(planes.nruns + 127) / 128, 128, 0, st>>>(runs, planes.nruns);
    return cudaGetLastError();
}

}  // namespace pic
