// adjoint.cu -- discrete adjoint of the EM-PIC timestep (reverse mode of
// exactly the forward arithmetic of push.cuh and fields.cu), for gradients
// of a scalar objective of the final particle state with respect to the
// particle weights (hence a density profile) and the laser amplitude a0.
//
// Reverse of one step n (forward: push/deposit -> B half -> E -> B half):
//   (i)   B^{n+1} = B^{n+1/2} - h curl_f E^{n+1} (+ antenna, t^{n+1}):
//         lamE -= h curl_b(m_B lamB)
//   (ii)  E^{n+1} = Mur(E^n, E~), E~ = E^n + dt (curl_b B^{n+1/2} - J) (+ antenna):
//         T = lamE on updated entries (+ Mur terms), lamB += dt curl_f(T),
//         lamJ = -dt T, lamE <- T on updated entries (+ Mur terms)
//   (iii) B^{n+1/2} = B^n - h curl_f E^n (+ antenna, t^n): as (i)
//   (iv)  particles: deposit transpose = gather of lamJ with the shape
//         derivatives; move, Boris and gather transposes; gather transpose
//         scatters into lamE, lamB.
// curl_b (backward differences) is the transpose of curl_f (forward
// differences) on the staggered grid; m_B masks the B entries the forward
// leaves frozen beyond an open end.  Particle adjoints live in arrays indexed
// by particle id, so the tile sort between steps does not matter.
#include <cstdint>
#include <utility>

#include "common.cuh"
#include "internal.h"

namespace pic {
namespace {

__device__ double laser_unit(const Run &r, double r2, double xi)
{
    // antenna field for a0 = 1 (the forward field is linear in a0)
    double dx = xi - r.t_peak;
    double env = exp(-2.0 * 0.69314718055994530942 * dx * dx / (r.fwhm * r.fwhm));
    return exp(-r2 / (r.waist * r.waist)) * env * cos(r.omega0 * dx);
}

__device__ double laser_r2_adj(const Run &r, int i, int j)
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

__device__ __forceinline__ double block_reduce(double v, double *sh)
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
    return t;
}

// B entries frozen by the forward beyond an open end (half-integer
// positions on the last axis at physical index nl-1).
template <int DIM>
__device__ __forceinline__ bool b_frozen(const Run &r, int comp, int il)
{
    if (!r.open_last || il != r.n[DIM - 1] - 1) return false;
    return DIM == 3 ? comp != 2 : comp != 1;
}

// (i)/(iii): lamE -= h curl_b(m_B lamB); antenna: lam_a0 += <lamB, dB/da0>.
// With mask (the (i) half, followed by (ii)): also T = newE = lamE on the
// entries the E update writes, 0 elsewhere (part 1 of (ii)).
template <int DIM>
__global__ void adj_b_kernel(const Run *__restrict__ run, AdjPtrs A, int origin, double t_b, int laser_on,
                             double *la0, int mask)
{
    const Run &r = *run;
    __shared__ double sh[32];
    double acc = 0.0;
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1, nl = r.n[DIM - 1];
    const float h = 0.5f * r.dt;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < r.ncell; idx += gridDim.x * blockDim.x) {
        const int i = idx % n0, j = (idx / n0) % n1, k = DIM == 3 ? idx / (n0 * n1) : 0;
        const int mx = (i == 0 ? n0 - 1 : i - 1) + n0 * (j + n1 * k);
        const int my = i + n0 * ((j == 0 ? n1 - 1 : j - 1) + n1 * k);
        const int mz = DIM == 3 ? i + n0 * (j + n1 * (k == 0 ? n2 - 1 : k - 1)) : idx;
        auto il_of = [&](int jj, int kk) {
            int s = (DIM == 3 ? kk : jj) - origin;
            return s < 0 ? s + nl : s;
        };
        const int il = il_of(j, k);
        const int il_my = il_of(j == 0 ? n1 - 1 : j - 1, k);
        const int il_mz = DIM == 3 ? il_of(j, k == 0 ? n2 - 1 : k - 1) : il;
        auto mb = [&](int comp, int at, int ill) { return b_frozen<DIM>(r, comp, ill) ? 0.f : A.lB[comp][at]; };
        const float bx = mb(0, idx, il), by = mb(1, idx, il), bz = mb(2, idx, il);
        const float dBz_dy = (bz - mb(2, my, il_my)) * r.inv_d[1], dBz_dx = (bz - mb(2, mx, il)) * r.inv_d[0];
        const float dBy_dx = (by - mb(1, mx, il)) * r.inv_d[0], dBx_dy = (bx - mb(0, my, il_my)) * r.inv_d[1];
        float dBy_dz = 0.f, dBx_dz = 0.f;
        if (DIM == 3) {
            dBy_dz = (by - mb(1, mz, il_mz)) * r.inv_d[2];
            dBx_dz = (bx - mb(0, mz, il_mz)) * r.inv_d[2];
        }
        const float e[3] = {A.lE[0][idx] - h * (dBz_dy - dBy_dz), A.lE[1][idx] - h * (dBx_dz - dBz_dx),
                            A.lE[2][idx] - h * (dBy_dx - dBx_dy)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A.lE[c][idx] = e[c];
            if (mask) {
                bool upd = true;
                if (r.open_last) {
                    const int t1 = DIM == 3 ? 1 : 2, nrm = DIM == 3 ? 2 : 1;
                    if ((c == 0 || c == t1) && (il == 0 || il == nl - 1)) upd = false;  // Mur-set tangential
                    if (c == nrm && il == nl - 1) upd = false;                          // zeroed normal
                }
                A.T[c][idx] = upd ? e[c] : 0.f;
                A.nE[c][idx] = upd ? e[c] : 0.f;
            }
        }
        if (laser_on && il == r.laser_plane - 1) {
            int bcomp;
            double sgn;
            if (DIM == 3) {
                bcomp = r.laser_pol == 0 ? 1 : 0;
                sgn = r.laser_pol == 0 ? 1.0 : -1.0;
            } else {
                bcomp = 2;
                sgn = -1.0;
            }
            acc += (double)A.lB[bcomp][idx] * sgn * (double)h * (double)r.inv_d[DIM - 1] *
                   laser_unit(r, laser_r2_adj(r, i, j), t_b);
        }
    }
    double t = block_reduce(acc, sh);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(la0, t);
}

// (ii) part 2: the Mur transposes (one thread per transverse position).
template <int DIM>
__global__ void adj_mur_kernel(const Run *__restrict__ run, AdjPtrs A, int origin)
{
    const Run &r = *run;
    if (!r.open_last) return;
    const int nl = r.n[DIM - 1];
    const int plane = r.ncell / nl;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= plane) return;
    const float dl = r.d[DIM - 1];
    const float coef = (r.dt - dl) / (r.dt + dl);
    auto at = [&](int pl) {
        int st = pl + origin;
        st = st >= nl ? st - nl : st;
        return q + plane * st;
    };
    const int tc[2] = {0, DIM == 3 ? 1 : 2};
    for (int t = 0; t < 2; ++t) {
        const int c = tc[t];
        const int c0 = at(0), c1 = at(1), cm = at(nl - 1), cm1 = at(nl - 2);
        // F0 = o1 + coef (F1 - o0);  Fm = om1 + coef (Fm1 - om)
        const float l0 = A.lE[c][c0], lm = A.lE[c][cm];
        A.T[c][c1] += coef * l0;
        A.nE[c][c1] += coef * l0 + l0;
        A.nE[c][c0] = -coef * l0;
        A.T[c][cm1] += coef * lm;
        A.nE[c][cm1] += coef * lm + lm;
        A.nE[c][cm] = -coef * lm;
    }
}

// (ii) part 3: lamB += dt curl_f(T); lamJ = -dt T; antenna a0 term.
template <int DIM>
__global__ void adj_e_curl_kernel(const Run *__restrict__ run, AdjPtrs A, int origin, double t_n, int laser_on,
                                  double *la0)
{
    const Run &r = *run;
    __shared__ double sh[32];
    double acc = 0.0;
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1, nl = r.n[DIM - 1];
    const float dt = r.dt;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < r.ncell; idx += gridDim.x * blockDim.x) {
        const int i = idx % n0, j = (idx / n0) % n1, k = DIM == 3 ? idx / (n0 * n1) : 0;
        const int cx = (i + 1 == n0 ? 0 : i + 1) + n0 * (j + n1 * k);
        const int cy = i + n0 * ((j + 1 == n1 ? 0 : j + 1) + n1 * k);
        const float tx = A.T[0][idx], ty = A.T[1][idx], tz = A.T[2][idx];
        const float dTz_dy = (A.T[2][cy] - tz) * r.inv_d[1], dTz_dx = (A.T[2][cx] - tz) * r.inv_d[0];
        const float dTy_dx = (A.T[1][cx] - ty) * r.inv_d[0], dTx_dy = (A.T[0][cy] - tx) * r.inv_d[1];
        float dTy_dz = 0.f, dTx_dz = 0.f;
        if (DIM == 3) {
            const int cz = i + n0 * (j + n1 * (k + 1 == n2 ? 0 : k + 1));
            dTy_dz = (A.T[1][cz] - ty) * r.inv_d[2];
            dTx_dz = (A.T[0][cz] - tx) * r.inv_d[2];
        }
        A.lB[0][idx] += dt * (dTz_dy - dTy_dz);
        A.lB[1][idx] += dt * (dTx_dz - dTz_dx);
        A.lB[2][idx] += dt * (dTy_dx - dTx_dy);
        A.lJ[0][idx] = -dt * tx;
        A.lJ[1][idx] = -dt * ty;
        A.lJ[2][idx] = -dt * tz;
        if (laser_on) {
            int il = (DIM == 3 ? k : j) - origin;
            il = il < 0 ? il + nl : il;
            if (il == r.laser_plane) {
                const double xi = t_n + 0.5 * r.dt_d + 0.5 * r.d_last_d;
                acc += (double)A.T[r.laser_pol][idx] * (double)dt * (double)r.inv_d[DIM - 1] *
                       laser_unit(r, laser_r2_adj(r, i, j), xi);
            }
        }
    }
    double t = block_reduce(acc, sh);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(la0, t);
}

// ---------------------------------------------------------------------------
// Per-particle adjoint.
// ---------------------------------------------------------------------------
// Node / half shapes with derivatives d w / d(offset).
template <int P>
struct ShapeD;
template <>
struct ShapeD<1> {
    static __device__ __forceinline__ void node(int c, float d, int &b, float *w, float *dw)
    {
        b = c;
        w[0] = 1.f - d;
        w[1] = d;
        dw[0] = -1.f;
        dw[1] = 1.f;
    }
    static __device__ __forceinline__ void half(int c, float d, int &b, float *w, float *dw)
    {
        bool hi = d >= 0.5f;
        float t = hi ? d - 0.5f : d + 0.5f;
        b = hi ? c : c - 1;
        w[0] = 1.f - t;
        w[1] = t;
        dw[0] = -1.f;
        dw[1] = 1.f;
    }
};
template <>
struct ShapeD<2> {
    static __device__ __forceinline__ void q(float t, float *w, float *dw)
    {
        float a = 0.5f - t, b = 0.5f + t;
        w[0] = 0.5f * a * a;
        w[1] = 0.75f - t * t;
        w[2] = 0.5f * b * b;
        dw[0] = -a;
        dw[1] = -2.f * t;
        dw[2] = b;
    }
    static __device__ __forceinline__ void node(int c, float d, int &b, float *w, float *dw)
    {
        int h = d >= 0.5f ? 1 : 0;
        b = c + h - 1;
        q(d - (float)h, w, dw);
    }
    static __device__ __forceinline__ void half(int c, float d, int &b, float *w, float *dw)
    {
        b = c - 1;
        q(d - 0.5f, w, dw);
    }
};
template <>
struct ShapeD<3> {
    static __device__ __forceinline__ void cub(float f, float *w, float *dw)
    {
        const float s = 1.f / 6.f;
        float g = 1.f - f, f2 = f * f, f3 = f2 * f;
        w[0] = g * g * g * s;
        w[1] = (4.f - 6.f * f2 + 3.f * f3) * s;
        w[2] = (1.f + 3.f * f + 3.f * f2 - 3.f * f3) * s;
        w[3] = f3 * s;
        dw[0] = -0.5f * g * g;
        dw[1] = -2.f * f + 1.5f * f2;
        dw[2] = 0.5f + f - 1.5f * f2;
        dw[3] = 0.5f * f2;
    }
    static __device__ __forceinline__ void node(int c, float d, int &b, float *w, float *dw)
    {
        b = c - 1;
        cub(d, w, dw);
    }
    static __device__ __forceinline__ void half(int c, float d, int &b, float *w, float *dw)
    {
        bool hi = d >= 0.5f;
        b = hi ? c - 1 : c - 2;
        cub(hi ? d - 0.5f : d + 0.5f, w, dw);
    }
};

struct GF {
    const float *p[6];
    int n0, n1, n2;
    __device__ __forceinline__ int at(int i, int j, int k) const
    {
        return wrapi(i, n0) + n0 * (wrapi(j, n1) + n1 * (n2 > 1 ? wrapi(k, n2) : 0));
    }
};

// Boris push keeping what its transpose needs.
struct BorisTape {
    float um[3], t[3], s[3], p[3], g, f;
};

__device__ __forceinline__ void cross(const float *a, const float *b, float *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void boris_fwd(float h, const float *e, const float *b, const float *u, float *out,
                                          BorisTape &tp)
{
    for (int a = 0; a < 3; ++a) tp.um[a] = fmaf(h, e[a], u[a]);
    tp.g = rsqrtf(1.f + tp.um[0] * tp.um[0] + tp.um[1] * tp.um[1] + tp.um[2] * tp.um[2]);
    for (int a = 0; a < 3; ++a) tp.t[a] = h * b[a] * tp.g;
    tp.f = 2.f * __frcp_rn(1.f + tp.t[0] * tp.t[0] + tp.t[1] * tp.t[1] + tp.t[2] * tp.t[2]);
    for (int a = 0; a < 3; ++a) tp.s[a] = tp.f * tp.t[a];
    float c[3];
    cross(tp.um, tp.t, c);
    for (int a = 0; a < 3; ++a) tp.p[a] = tp.um[a] + c[a];
    cross(tp.p, tp.s, c);
    for (int a = 0; a < 3; ++a) out[a] = fmaf(h, e[a], tp.um[a] + c[a]);
}

// Transpose of boris_fwd: lam_out -> lam_u, lam_e, lam_b.
__device__ __forceinline__ void boris_vjp(float h, const float *b, const BorisTape &tp, const float *lo, float *lu,
                                          float *le, float *lb)
{
    float lum[3], lp[3], ls[3], lt[3], c[3];
    for (int a = 0; a < 3; ++a) {
        le[a] = h * lo[a];
        lum[a] = lo[a];  // out = um + p x s + h e
    }
    cross(tp.s, lo, lp);  // d(p x s)/dp^T lo = s x lo
    cross(lo, tp.p, ls);  // d(p x s)/ds^T lo = lo x p
    // p = um + um x t
    cross(tp.t, lp, c);
    for (int a = 0; a < 3; ++a) lum[a] += lp[a] + c[a];
    cross(lp, tp.um, lt);
    // s = f t, f = 2/(1+|t|^2), df/dt = -f^2 t
    const float lf = ls[0] * tp.t[0] + ls[1] * tp.t[1] + ls[2] * tp.t[2];
    for (int a = 0; a < 3; ++a) lt[a] += tp.f * ls[a] - lf * tp.f * tp.f * tp.t[a];
    // t = h b g, g = (1+|um|^2)^(-1/2), dg/dum = -g^3 um
    float lg = 0.f;
    for (int a = 0; a < 3; ++a) {
        lb[a] = h * tp.g * lt[a];
        lg += h * b[a] * lt[a];
    }
    const float g3 = tp.g * tp.g * tp.g;
    for (int a = 0; a < 3; ++a) lum[a] -= lg * g3 * tp.um[a];
    // um = u + h e
    for (int a = 0; a < 3; ++a) {
        lu[a] = lum[a];
        le[a] += h * lum[a];
    }
}

// Recorded fields / current adjoint read through global memory (absolute,
// wrapped indices) or from a tile staged in shared memory (tile-relative).
struct GlobalRead {
    const float *p[9];  // E0..2, B0..2 (recorded) then lamJ0..2
    int n0, n1, n2;
    __device__ __forceinline__ float operator()(int comp, int i, int j, int k) const
    {
        return __ldg(p[comp] + wrapi(i, n0) + n0 * (wrapi(j, n1) + n1 * (n2 > 1 ? wrapi(k, n2) : 0)));
    }
};
// The same with the tile geometry fixed at compile time (immediate offsets).
template <int FV, int FS0, int FS01, int FH0, int FH1, int FH2, int JV, int JS0, int JS01, int JH0, int JH1, int JH2>
struct SmemReadC {
    const float *f;
    const float *l;
    __device__ __forceinline__ float operator()(int comp, int i, int j, int k) const
    {
        return comp < 6 ? f[comp * FV + (i + FH0) + FS0 * (j + FH1) + FS01 * (k + FH2)]
                        : l[(comp - 6) * JV + (i + JH0) + JS0 * (j + JH1) + JS01 * (k + JH2)];
    }
};
struct SmemRead {
    const float *f;  // 6 field components, region fvol each
    const float *l;  // 3 current-adjoint components, region jvol each
    int fvol, fh0, fh1, fh2, fs0, fs01;
    int jvol, jh0, jh1, jh2, js0, js01;
    __device__ __forceinline__ float operator()(int comp, int i, int j, int k) const
    {
        return comp < 6 ? f[comp * fvol + (i + fh0) + fs0 * (j + fh1) + fs01 * (k + fh2)]
                        : l[(comp - 6) * jvol + (i + jh0) + js0 * (j + jh1) + js01 * (k + jh2)];
    }
};

// Inputs of one recorded particle's adjoint: its recorded state and the
// adjoints of its state after the step (slot order).
struct AdjIn {
    int32_t cell;
    float d[3], u[3], w;
    float lx[3], lu[3];
    double lw;  // accumulated weight adjoint of the slot
};

template <int DIM>
__device__ __forceinline__ void adj_load(const TrajStep &ts, const AdjPtrs &A, long long s, AdjIn &in)
{
    in.cell = ts.cell[s];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        in.d[a] = a < DIM ? ts.off[a][s] : 0.f;
        in.lx[a] = a < DIM ? A.sx[a][s] : 0.f;
        in.u[a] = ts.u[a][s];
        in.lu[a] = A.su[a][s];
    }
    in.w = ts.w[s];
    in.lw = A.sw[s];
}

// One recorded particle's adjoint.  c: cell in the reader's frame; org:
// offset from that frame to absolute cells (scatter and absorption use
// absolute cells); rd(comp 0..5, ...) reads the recorded fields,
// rd(6 + comp, ...) the current adjoint.
template <int DIM, int P, class RD>
__device__ __forceinline__ void adj_one(const Run &r, const AdjPtrs &A, const TrajStep &ts, long long s,
                                        const AdjIn &in, int origin, const int *c, const int *org, const RD &rd)
{
    const int nl = r.n[DIM - 1];
    float d[3] = {0.f, 0.f, 0.f}, u[3];
#pragma unroll
    for (int a = 0; a < DIM; ++a) d[a] = in.d[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = in.u[a];
    const float w = in.w;
    const GF gf{{ts.E[0], ts.E[1], ts.E[2], ts.B[0], ts.B[1], ts.B[2]}, r.n[0], r.n[1], DIM == 3 ? r.n[2] : 1};
    const int ox = org[0], oy = org[1], oz = org[2];
    // --- forward recompute: shapes and gather with position derivatives ---
    int bn[3] = {0, 0, 0}, bh[3] = {0, 0, 0};
    float wn[DIM][P + 1], wh[DIM][P + 1], dwn[DIM][P + 1], dwh[DIM][P + 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        ShapeD<P>::node(c[a], d[a], bn[a], wn[a], dwn[a]);
        ShapeD<P>::half(c[a], d[a], bh[a], wh[a], dwh[a]);
    }
    // half-integer flags per component (E0 E1 E2 B0 B1 B2) and axis
    const unsigned hxm = 0x31u, hym = 0x2Au, hzm = 0x1Cu;
    float eb[6], deb[6][DIM];
#pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        const bool hx = (hxm >> comp) & 1u, hy = (hym >> comp) & 1u, hz = (hzm >> comp) & 1u;
        const int b0 = hx ? bh[0] : bn[0], b1 = hy ? bh[1] : bn[1], b2 = hz ? bh[2] : bn[2];
        float v = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int kc = 0; kc < (DIM == 3 ? P + 1 : 1); ++kc) {
            const float wz = DIM == 3 ? (hz ? wh[DIM - 1][kc] : wn[DIM - 1][kc]) : 1.f;
            const float dwz = DIM == 3 ? (hz ? dwh[DIM - 1][kc] : dwn[DIM - 1][kc]) : 0.f;
#pragma unroll
            for (int kb = 0; kb <= P; ++kb) {
                const float wy = hy ? wh[1][kb] : wn[1][kb], dwy = hy ? dwh[1][kb] : dwn[1][kb];
                const float wyz = wy * wz;
                float sx = 0.f, sdx = 0.f;
#pragma unroll
                for (int ka = 0; ka <= P; ++ka) {
                    const float wx = hx ? wh[0][ka] : wn[0][ka], dwx = hx ? dwh[0][ka] : dwn[0][ka];
                    const float F = rd(comp, b0 + ka, b1 + kb, b2 + kc);
                    sx = fmaf(wx, F, sx);
                    sdx = fmaf(dwx, F, sdx);
                }
                v = fmaf(wyz, sx, v);
                g0 = fmaf(wyz, sdx, g0);
                g1 = fmaf(dwy * wz, sx, g1);
                g2 = fmaf(wy * dwz, sx, g2);
            }
        }
        eb[comp] = v;
        deb[comp][0] = g0;
        deb[comp][1] = g1;
        if (DIM == 3) deb[comp][DIM - 1] = g2;
    }
    BorisTape tp;
    float un[3];
    boris_fwd(r.qm_half_dt, eb, eb + 3, u, un, tp);
    const float ig = rsqrtf(1.f + un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
    float d1[3] = {0.f, 0.f, 0.f};
    int k[3] = {0, 0, 0};
    bool ok = true;
    for (int a = 0; a < DIM; ++a) {
        float nd = d[a] + r.dt_over_d[a] * un[a] * ig;
        ok = ok && nd > -1.f && nd < 2.f;
        float kk = floorf(nd);
        nd = nd - kk;
        if (nd >= 1.f) {
            nd = 0.f;
            kk += 1.f;
        }
        d1[a] = nd;
        k[a] = (int)kk;
    }
    if (!ok) return;
    bool absorbed = false;
    if (r.open_last) {
        int cl = wrapi(c[DIM - 1] + org[DIM - 1] + k[DIM - 1], nl) - origin;
        cl = cl < 0 ? cl + nl : cl;
        absorbed = cl < r.margin || cl >= nl - r.margin;
    }
    // --- adjoint inputs: state adjoints of x^{n+1}, u^{n+1/2} ---
    float lxn[3] = {0.f, 0.f, 0.f}, lun[3] = {0.f, 0.f, 0.f};
    if (!absorbed) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) lxn[a] = in.lx[a];
#pragma unroll
        for (int a = 0; a < 3; ++a) lun[a] = in.lu[a];
    }
    // --- deposit transpose (Esirkepov window, per unit weight) ---
    constexpr int W = P + 2;
    float S0[DIM][W], S1[DIM][W], dS0[DIM][W], dS1[DIM][W];
    int wb[3] = {0, 0, 0};
    bool moved[3] = {false, false, false};  // nearest node changed along the axis
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int q = 0; q < W; ++q) S0[a][q] = S1[a][q] = dS0[a][q] = dS1[a][q] = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int bo, bnw;
        float so[P + 1], sn[P + 1], dso[P + 1], dsn[P + 1];
        ShapeD<P>::node(c[a], d[a], bo, so, dso);
        ShapeD<P>::node(c[a] + k[a], d1[a], bnw, sn, dsn);
        const int sh = bnw - bo;
        moved[a] = sh != 0;
        wb[a] = sh < 0 ? bnw : bo;
        const int oo = sh < 0 ? 1 : 0, on = sh > 0 ? 1 : 0;
#pragma unroll
        for (int q = 0; q <= P; ++q) {
            // compile-time q; the runtime offset selects between two slots
            if (oo) {
                S0[a][q + 1] = so[q];
                dS0[a][q + 1] = dso[q];
            } else {
                S0[a][q] = so[q];
                dS0[a][q] = dso[q];
            }
            if (on) {
                S1[a][q + 1] = sn[q];
                dS1[a][q + 1] = dsn[q];
            } else {
                S1[a][q] = sn[q];
                dS1[a][q] = dsn[q];
            }
        }
    }
    float As[DIM][W], DS[DIM][W], Pr[DIM][W];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        float run_ = 0.f;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            DS[a][q] = S1[a][q] - S0[a][q];
            As[a][q] = S0[a][q] + 0.5f * DS[a][q];
            run_ += DS[a][q];
            Pr[a][q] = run_;
        }
        // as in the forward deposit: without a node change the last prefix
        // is exactly zero (and carries no derivative)
        if (!moved[a]) Pr[a][W - 2] = 0.f;
    }
    // the forward skips the last window node of an axis along which no lane
    // of the warp changed node (all its terms are zero); so does the adjoint
    const unsigned act = __activemask();
    bool fa[3] = {true, true, true};
#pragma unroll
    for (int a = 0; a < DIM; ++a) fa[a] = __any_sync(act, moved[a]);
    const float q_ = r.q;
    const float vz = un[2] * ig;
    float gA[DIM][W], gD[DIM][W];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int q = 0; q < W; ++q) gA[a][q] = gD[a][q] = 0.f;
    float lw = 0.f, gvz = 0.f;
    auto lam = [&](int comp, int i, int j, int kk) { return rd(6 + comp, i, j, kk); };
    if (DIM == 2) {
        const float cx = -q_ * r.d_over_dt[0], cy = -q_ * r.d_over_dt[1];
        float Rx[W], Ry[W];
#pragma unroll
        for (int q = 0; q < W; ++q) Rx[q] = Ry[q] = 0.f;
#pragma unroll
        for (int qb = 0; qb < W; ++qb)
#pragma unroll
            for (int qa = 0; qa < W; ++qa) {
                if ((qb == W - 1 && !fa[1]) || (qa == W - 1 && !fa[0])) continue;
                const int i = wb[0] + qa, j = wb[1] + qb;
                if (qa < W - 1 && !(qa == W - 2 && !fa[0])) {  // J_x = cx P_x A_y
                    const float L = lam(0, i, j, 0);
                    lw += L * cx * Pr[0][qa] * As[1][qb];
                    Rx[qa] += L * As[1][qb];
                    gA[1][qb] += w * cx * L * Pr[0][qa];
                }
                if (qb < W - 1 && !(qb == W - 2 && !fa[1])) {  // J_y = cy P_y A_x
                    const float L = lam(1, i, j, 0);
                    lw += L * cy * Pr[1][qb] * As[0][qa];
                    Ry[qb] += L * As[0][qa];
                    gA[0][qa] += w * cy * L * Pr[1][qb];
                }
                {  // J_z = q vz (A_x A_y + DS_x DS_y / 12)
                    const float L = lam(2, i, j, 0);
                    const float fz = As[0][qa] * As[1][qb] + DS[0][qa] * DS[1][qb] * (1.f / 12.f);
                    lw += L * q_ * vz * fz;
                    gvz += w * q_ * L * fz;
                    gA[0][qa] += w * q_ * vz * L * As[1][qb];
                    gA[1][qb] += w * q_ * vz * L * As[0][qa];
                    gD[0][qa] += w * q_ * vz * L * DS[1][qb] * (1.f / 12.f);
                    gD[1][qb] += w * q_ * vz * L * DS[0][qa] * (1.f / 12.f);
                }
            }
        // prefix transposes: d/dDS[a'] of sum_a R[a] P[a] = sum_{a>=a'} R[a]
        // (a prefix forced to zero passes no derivative)
        if (!moved[0]) Rx[W - 2] = 0.f;
        if (!moved[1]) Ry[W - 2] = 0.f;
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int q = W - 2; q >= 0; --q) {
            sx += Rx[q];
            sy += Ry[q];
            gD[0][q] += w * cx * sx;
            gD[1][q] += w * cy * sy;
        }
    } else {
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const int a = comp % DIM, b = (comp + 1) % DIM, cc = (comp + 2) % DIM;
            const float coef = -q_ * r.d_over_dt[a];
            float R[W];
            for (int q = 0; q < W; ++q) R[q] = 0.f;
            for (int qc = 0; qc < W; ++qc)
                for (int qb = 0; qb < W; ++qb) {
                    if ((qc == W - 1 && !fa[cc]) || (qb == W - 1 && !fa[b])) continue;
                    const float fac = As[b][qb] * As[cc][qc] + DS[b][qb] * DS[cc][qc] * (1.f / 12.f);
                    for (int qa = 0; qa < W - 1; ++qa) {
                        if (qa == W - 2 && !fa[a]) continue;
                        int q3[3];
                        q3[a] = qa;
                        q3[b] = qb;
                        q3[cc] = qc;
                        const float L = lam(comp, wb[0] + q3[0], wb[1] + q3[1], wb[2] + q3[2]);
                        lw += L * coef * Pr[a][qa] * fac;
                        R[qa] += L * fac;
                        const float lp = w * coef * L * Pr[a][qa];
                        gA[b][qb] += lp * As[cc][qc];
                        gA[cc][qc] += lp * As[b][qb];
                        gD[b][qb] += lp * DS[cc][qc] * (1.f / 12.f);
                        gD[cc][qc] += lp * DS[b][qb] * (1.f / 12.f);
                    }
                }
            if (!moved[a]) R[W - 2] = 0.f;
            float sacc = 0.f;
            for (int q = W - 2; q >= 0; --q) {
                sacc += R[q];
                gD[a][q] += w * coef * sacc;
            }
        }
    }
    // A = S0 + DS/2 = (S0 + S1)/2, DS = S1 - S0  ->  d/dS0 = gA/2 - gD, d/dS1 = gA/2 + gD
    float lxo[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        float go = 0.f, gn = 0.f;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            go += (0.5f * gA[a][q] - gD[a][q]) * dS0[a][q];
            gn += (0.5f * gA[a][q] + gD[a][q]) * dS1[a][q];
        }
        lxo[a] = go;
        lxn[a] += gn;
    }
    // --- move transpose: x1 = x0 + (dt/d) u/gamma ; vz = u_z / gamma ---
    float lut[3] = {lun[0], lun[1], lun[2]};
    float gv[3] = {0.f, 0.f, 0.f};  // d L / d v_a with v = u/gamma
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        gv[a] += lxn[a] * r.dt_over_d[a];
        lxo[a] += lxn[a];
    }
    if (DIM == 2) gv[2] += gvz;
    {
        const float vv = gv[0] * un[0] + gv[1] * un[1] + gv[2] * un[2];
        const float ig3 = ig * ig * ig;
        for (int a = 0; a < 3; ++a) lut[a] += gv[a] * ig - vv * un[a] * ig3;
    }
    // --- Boris transpose ---
    float lu0[3], le[3], lb[3];
    boris_vjp(r.qm_half_dt, eb + 3, tp, lut, lu0, le, lb);
    const float lebs[6] = {le[0], le[1], le[2], lb[0], lb[1], lb[2]};
    // --- gather transpose: positions and scatter into lamE, lamB ---
#pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        const float L = lebs[comp];
        for (int a = 0; a < DIM; ++a) lxo[a] += L * deb[comp][a];
        if (L == 0.f) continue;
        const bool hx = (hxm >> comp) & 1u, hy = (hym >> comp) & 1u, hz = (hzm >> comp) & 1u;
        const int b0 = hx ? bh[0] : bn[0], b1 = hy ? bh[1] : bn[1], b2 = hz ? bh[2] : bn[2];
        float *dst = comp < 3 ? A.lE[comp] : A.lB[comp - 3];
#pragma unroll
        for (int kc = 0; kc < (DIM == 3 ? P + 1 : 1); ++kc) {
            const float wz = DIM == 3 ? (hz ? wh[DIM - 1][kc] : wn[DIM - 1][kc]) : 1.f;
#pragma unroll
            for (int kb = 0; kb <= P; ++kb) {
                const float wy = hy ? wh[1][kb] : wn[1][kb];
#pragma unroll
                for (int ka = 0; ka <= P; ++ka) {
                    const float wx = hx ? wh[0][ka] : wn[0][ka];
                    atomicAdd(dst + gf.at(b0 + ka + ox, b1 + kb + oy, b2 + kc + oz), L * wx * wy * wz);
                }
            }
        }
    }
    // outputs: in place, or (after a sort) at the slot the particle had before it
    if (ts.src) {
        const long long o = ts.src[s];
        for (int a = 0; a < DIM; ++a) A.ox[a][o] = lxo[a];
        for (int a = 0; a < 3; ++a) A.ou[a][o] = lu0[a];
        A.ow[o] = in.lw + (double)lw;
    } else {
        for (int a = 0; a < DIM; ++a) A.sx[a][s] = lxo[a];
        for (int a = 0; a < 3; ++a) A.su[a][s] = lu0[a];
        A.sw[s] = in.lw + (double)lw;
    }
}

template <int DIM>
__device__ __forceinline__ bool adj_live(const Run &r, int32_t pc, int origin, int *c)
{
    if (pc < 0) return false;
    unpack_cell(r, pc, c[0], c[1], c[2]);
    if (r.open_last) {
        const int nl = r.n[DIM - 1];
        int pl = c[DIM - 1] - origin;
        pl = pl < 0 ? pl + nl : pl;
        if (pl < r.margin || pl >= nl - r.margin) return false;  // removed before this push
    }
    return true;
}

// Flat form: one thread per recorded slot, everything through global memory.
template <int DIM, int P>
__global__ void __launch_bounds__(128, 3) adj_particles_kernel(const Run *__restrict__ run, AdjPtrs A, TrajStep ts,
                                                               int origin)
{
    const Run &r = *run;
    const long long s = ts.first + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ts.n) return;
    int c[3] = {0, 0, 0};
    if (!adj_live<DIM>(r, ts.cell[s], origin, c)) return;
    AdjIn in;
    adj_load<DIM>(ts, A, s, in);
    const GlobalRead g{{ts.E[0], ts.E[1], ts.E[2], ts.B[0], ts.B[1], ts.B[2], A.lJ[0], A.lJ[1], A.lJ[2]},
                       r.n[0], r.n[1], DIM == 3 ? r.n[2] : 1};
    const int org[3] = {0, 0, 0};
    adj_one<DIM, P>(r, A, ts, s, in, origin, c, org, g);
}

// Tiled form: nsplit CTAs per tile of the sort recorded with the step (each
// takes every nsplit-th group of blockDim particles); the tile's recorded
// fields and current adjoint (plus halos wide enough for particles within
// `drift` cells of the tile) are staged in shared memory.
// TX > 0: tile TX x TY (x TZ) with drift DR fixed at compile time (constant
// shared-memory strides); TX = 0: the run's tile geometry at run time.
template <int DIM, int P, int TX, int TY, int TZ, int DR>
__global__ void __launch_bounds__(128, 3) adj_particles_tiled_kernel(const Run *__restrict__ run, AdjPtrs A,
                                                                     TrajStep ts, int origin, int nsplit)
{
    extern __shared__ float sm[];
    const Run &r = *run;
    const int t = blockIdx.x / nsplit, part = blockIdx.x - t * nsplit;
    const long long p0 = ts.tile_off[t], p1 = ts.tile_off[t + 1];
    if (p0 >= p1) return;
    constexpr bool CT = TX > 0;
    const int D = CT ? DR : r.drift;
    const int n0 = r.n[0], n1 = r.n[1], n2 = DIM == 3 ? r.n[2] : 1;
    int org[3] = {0, 0, 0}, T[3] = {1, 1, 1}, fh[3] = {0, 0, 0}, fs[3] = {1, 1, 1}, jh[3] = {0, 0, 0},
        js[3] = {1, 1, 1};
    org[0] = (t % r.nt[0]) << r.tlog[0];
    org[1] = ((t / r.nt[0]) % r.nt[1]) << r.tlog[1];
    if (DIM == 3) org[2] = (t / (r.nt[0] * r.nt[1])) << r.tlog[2];
    for (int a = 0; a < DIM; ++a) {
        T[a] = CT ? (a == 0 ? TX : (a == 1 ? TY : TZ)) : 1 << r.tlog[a];
        fh[a] = D + Reach<P>::GLO;
        fs[a] = T[a] + 2 * D + Reach<P>::GLO + Reach<P>::GHI;
        jh[a] = D + Reach<P>::DLO;
        js[a] = T[a] + 2 * D + Reach<P>::DLO + Reach<P>::DHI;
    }
    const int fvol = fs[0] * fs[1] * fs[2], jvol = js[0] * js[1] * js[2];
    float *F = sm, *L = sm + 6 * fvol;
    for (int l = threadIdx.x; l < fvol; l += blockDim.x) {
        const int lx = l % fs[0], ly = (l / fs[0]) % fs[1], lz = l / (fs[0] * fs[1]);
        const int g = modi(org[0] - fh[0] + lx, n0) +
                      n0 * (modi(org[1] - fh[1] + ly, n1) + n1 * (DIM == 3 ? modi(org[2] - fh[2] + lz, n2) : 0));
        for (int c = 0; c < 3; ++c) {
            F[c * fvol + l] = __ldg(ts.E[c] + g);
            F[(3 + c) * fvol + l] = __ldg(ts.B[c] + g);
        }
    }
    int lj_any = 0;  // some current adjoint in reach of the tile is nonzero
    for (int l = threadIdx.x; l < jvol; l += blockDim.x) {
        const int lx = l % js[0], ly = (l / js[0]) % js[1], lz = l / (js[0] * js[1]);
        const int g = modi(org[0] - jh[0] + lx, n0) +
                      n0 * (modi(org[1] - jh[1] + ly, n1) + n1 * (DIM == 3 ? modi(org[2] - jh[2] + lz, n2) : 0));
        for (int c = 0; c < 3; ++c) {
            const float v = __ldg(A.lJ[c] + g);
            L[c * jvol + l] = v;
            lj_any |= v != 0.f;
        }
    }
    lj_any = __syncthreads_or(lj_any);
    const SmemRead sr{F, L, fvol, fh[0], fh[1], fh[2], fs[0], fs[0] * fs[1],
                      jvol, jh[0], jh[1], jh[2], js[0], js[0] * js[1]};
    constexpr int CTX = TX > 0 ? TX : 1, CTY = TX > 0 ? TY : 1, CTZ = DIM == 3 && TX > 0 ? TZ : 1;
    constexpr int GL = Reach<P>::GLO, GH = Reach<P>::GHI, DL = Reach<P>::DLO, DH = Reach<P>::DHI;
    constexpr int FS0 = CTX + 2 * DR + GL + GH, FS1 = CTY + 2 * DR + GL + GH, FS2 = DIM == 3 ? CTZ + 2 * DR + GL + GH : 1;
    constexpr int JS0 = CTX + 2 * DR + DL + DH, JS1 = CTY + 2 * DR + DL + DH, JS2 = DIM == 3 ? CTZ + 2 * DR + DL + DH : 1;
    const SmemReadC<FS0 * FS1 * FS2, FS0, FS0 * FS1, DR + GL, DR + GL, DIM == 3 ? DR + GL : 0, JS0 * JS1 * JS2, JS0,
                    JS0 * JS1, DR + DL, DR + DL, DIM == 3 ? DR + DL : 0>
        src_c{F, L};
    const GlobalRead g{{ts.E[0], ts.E[1], ts.E[2], ts.B[0], ts.B[1], ts.B[2], A.lJ[0], A.lJ[1], A.lJ[2]},
                       n0, n1, n2};
    const int zero[3] = {0, 0, 0};
    // the next particle's inputs are loaded before the current one is done
    AdjIn cur, nxt;
    const long long stride = (long long)blockDim.x * nsplit;
    long long s = p0 + (long long)part * blockDim.x + threadIdx.x;
    if (s < p1) adj_load<DIM>(ts, A, s, cur);
    for (; s < p1; s += stride) {
        if (s + stride < p1) adj_load<DIM>(ts, A, s + stride, nxt);
        int c[3] = {0, 0, 0};
        bool skip = !adj_live<DIM>(r, cur.cell, origin, c);
        if (!skip && !lj_any) {
            // zero state adjoints and a zero current adjoint give zero outputs
            bool zero = cur.lu[0] == 0.f && cur.lu[1] == 0.f && cur.lu[2] == 0.f;
#pragma unroll
            for (int a = 0; a < DIM; ++a) zero = zero && cur.lx[a] == 0.f;
            skip = zero;
            // the accumulated weight adjoint still follows the particle
            if (skip && ts.src) A.ow[ts.src[s]] = cur.lw;
        }
        if (!skip) {
            int rel[3] = {0, 0, 0};
            bool fast = true;
            for (int a = 0; a < DIM; ++a) {
                int v = c[a] - org[a];
                if (v < -D) v += r.n[a];
                else if (v >= T[a] + D) v -= r.n[a];
                rel[a] = v;
                fast = fast && v >= -D && v < T[a] + D;
            }
            if (fast) {
                if constexpr (CT) adj_one<DIM, P>(r, A, ts, s, cur, origin, rel, org, src_c);
                else adj_one<DIM, P>(r, A, ts, s, cur, origin, rel, org, sr);
            } else {
                adj_one<DIM, P>(r, A, ts, s, cur, origin, c, zero, g);
            }
        }
        cur = nxt;
    }
}

__global__ void adj_perm_kernel(AdjPtrs A, const int32_t *__restrict__ id, long long n, long long nid, int dim,
                                int to_slots)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int i = id[s];
        if (i < 0 || i >= nid) continue;
        if (to_slots) {
            for (int a = 0; a < dim; ++a) A.sx[a][s] = A.lx[a][i];
            for (int a = 0; a < 3; ++a) A.su[a][s] = A.lu[a][i];
            A.sw[s] = A.lw[i];
        } else {
            for (int a = 0; a < dim; ++a) A.lx[a][i] = A.sx[a][s];
            for (int a = 0; a < 3; ++a) A.lu[a][i] = A.su[a][s];
            A.lw[i] = A.sw[s];
        }
    }
}

// Transpose of a moving-window shift at the end of a step, applied before
// that step's field and particle transposes.  The forward set E and B on the
// new front plane (storage index store_plane of the last axis) to zero, so
// their adjoints there are zero; and it appended a cold layer of particles
// at slots slot0 + j with ids id0 + j, whose positions and momenta are
// constants: only their weights depend on the parameters, so their weight
// adjoints go to id order and their slot adjoints are cleared (slot0 < 0: the
// layer's adjoints are already in id order, at a segment's last step).
__global__ void adj_window_kernel(AdjPtrs A, int plane, int store_plane, long long slot0, long long count,
                                  long long id0, long long nid)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < plane) {
        const long long idx = q + (long long)plane * store_plane;
        for (int c = 0; c < 3; ++c) {
            A.lE[c][idx] = 0.f;
            A.lB[c][idx] = 0.f;
        }
    }
    if (slot0 >= 0 && q < count) {
        const long long slot = slot0 + q, id = id0 + q;
        if (id < nid) A.lw[id] = A.sw[slot];
        for (int a = 0; a < 3; ++a) {
            if (A.sx[a]) A.sx[a][slot] = 0.f;
            A.su[a][slot] = 0.f;
        }
        A.sw[slot] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Objective: L = sum w K sigma / sum w sigma, K = m (gamma - 1),
// sigma(z) = logistic((z - z_lo)/width) logistic((z_hi - z)/width), z the
// last-axis position in cells (window frame).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float logistic(float x) { return 1.f / (1.f + __expf(-x)); }

__device__ __forceinline__ bool obj_particle(const Run &r, const ParticleBuf &pb, long long i, int origin,
                                             const ObjArgs &o, float &w, float &z, float &sig, float &dsig)
{
    const int32_t pc = pb.cell[i];
    if (pc < 0) return false;
    int c[3];
    unpack_cell(r, pc, c[0], c[1], c[2]);
    const int nl = r.n[r.dim - 1];
    int cl = c[r.dim - 1] - (r.open_last ? origin : 0);
    cl = cl < 0 ? cl + nl : cl;
    if (r.open_last && (cl < r.margin || cl >= nl - r.margin)) return false;
    z = (float)cl + pb.off[r.dim - 1][i];
    const float a = logistic((z - o.z_lo) / o.width), b = logistic((o.z_hi - z) / o.width);
    sig = a * b;
    dsig = (a * (1.f - a) * b - a * b * (1.f - b)) / o.width;
    w = pb.w ? pb.w[i] : r.w_const;
    return true;
}

__global__ void obj_reduce_kernel(const Run *__restrict__ run, int origin, ObjArgs o, double *out)
{
    const Run &r = *run;
    const RunState &s = *r.state;
    const ParticleBuf pb = r.P[s.buf];
    __shared__ double sh[32];
    double num = 0.0, den = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < s.n_total;
         i += (long long)gridDim.x * blockDim.x) {
        float w, z, sig, dsig;
        if (!obj_particle(r, pb, i, origin, o, w, z, sig, dsig)) continue;
        const double ux = pb.u[0][i], uy = pb.u[1][i], uz = pb.u[2][i];
        const double K = (double)r.m * (sqrt(1.0 + ux * ux + uy * uy + uz * uz) - 1.0);
        num += (double)w * K * sig;
        den += (double)w * sig;
    }
    double a = block_reduce(num, sh), b = block_reduce(den, sh);
    if (threadIdx.x == 0) {
        atomicAdd(out + 0, a);
        atomicAdd(out + 1, b);
    }
}

__global__ void obj_seed_kernel(const Run *__restrict__ run, int origin, ObjArgs o, const double *red, AdjPtrs A)
{
    const Run &r = *run;
    const RunState &s = *r.state;
    const ParticleBuf pb = r.P[s.buf];
    const double den = red[1];
    const double L = den > 0.0 ? red[0] / den : 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < s.n_total;
         i += (long long)gridDim.x * blockDim.x) {
        float w, z, sig, dsig;
        if (!obj_particle(r, pb, i, origin, o, w, z, sig, dsig)) continue;
        const int id = pb.id[i];
        if (id < 0 || id >= r.adj_nid) continue;
        const float ux = pb.u[0][i], uy = pb.u[1][i], uz = pb.u[2][i];
        const float gam = sqrtf(1.f + ux * ux + uy * uy + uz * uz);
        const float K = r.m * (gam - 1.f);
        const float sc = (float)(den > 0.0 ? 1.0 / den : 0.0);
        A.lu[0][id] = w * sig * r.m * ux / gam * sc;
        A.lu[1][id] = w * sig * r.m * uy / gam * sc;
        A.lu[2][id] = w * sig * r.m * uz / gam * sc;
        for (int a = 0; a < r.dim - 1; ++a) A.lx[a][id] = 0.f;
        A.lx[r.dim - 1][id] = w * dsig * (K - (float)L) * sc;
        A.lw[id] = (double)(sig * (K - (float)L) * sc);
    }
}

// dL/dknot_k = sum_id dL/dw_id * phi_k(z_birth) / ppc_total (hat functions on
// equally spaced knots over [z0, z1], clamped outside).
__global__ void knots_kernel(const double *lw, const float *zb, long long n, int n_knots, double z0, double z1,
                             double ppc_t, double *out)
{
    __shared__ double acc[1024];  // per-block partial sums, one atomic per knot per block
    for (int k = threadIdx.x; k < n_knots; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const double g = lw[id] / ppc_t;
        if (g == 0.0) continue;
        double f = ((double)zb[id] - z0) / (z1 - z0) * (n_knots - 1);
        if (n_knots == 1 || f <= 0.0) {
            atomicAdd(acc, g);
        } else if (f >= n_knots - 1) {
            atomicAdd(acc + n_knots - 1, g);
        } else {
            const int i = (int)floor(f);
            const double t = f - i;
            atomicAdd(acc + i, g * (1.0 - t));
            atomicAdd(acc + i + 1, g * t);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_knots; k += blockDim.x)
        if (acc[k] != 0.0) atomicAdd(out + k, acc[k]);
}

// weights and birth positions by id of the loaded particles (the load
// order, before any sort; the window's injection writes those of the ids it
// creates)
__global__ void adj_init_kernel(const Run *__restrict__ run, float *wid, float *zb, long long n, long long nid)
{
    const Run &r = *run;
    const RunState &s = *r.state;
    const ParticleBuf pb = r.P[s.buf];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n && i < s.n_total;
         i += (long long)gridDim.x * blockDim.x) {
        const int id = pb.id[i];
        if (id < 0 || id >= nid) continue;
        wid[id] = pb.w ? pb.w[i] : r.w_const;
        int c[3];
        unpack_cell(r, pb.cell[i] < 0 ? 0 : pb.cell[i], c[0], c[1], c[2]);
        zb[id] = ((float)c[r.dim - 1] + pb.off[r.dim - 1][i]) * (float)r.d_last_d;
    }
}

// Copy the live buffer's first n slots to / from a side buffer (the
// current buffer index is read from the device state).
// Copy of the particle state to (restore = 0) or from (restore = 1) a
// record; each thread moves 4 consecutive slots with 16-byte accesses (the
// buffers are 256-byte aligned), the last n % 4 slots one by one.
template <int DIM>
__device__ __forceinline__ void copy4(int32_t *dc, float *const *doff, float *const *du, float *dw, int32_t *did,
                                      const int32_t *sc, const float *const *soff, const float *const *su,
                                      const float *sw, const int32_t *sid, long long i, long long n,
                                      long long n_live, bool fill_dead, bool vec)
{
    if (vec && i + 3 < n) {
        int4 c = *reinterpret_cast<const int4 *>(sc + i);
        if (fill_dead) {
            c.x = i < n_live ? c.x : -1;
            c.y = i + 1 < n_live ? c.y : -1;
            c.z = i + 2 < n_live ? c.z : -1;
            c.w = i + 3 < n_live ? c.w : -1;
        }
        *reinterpret_cast<int4 *>(dc + i) = c;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            *reinterpret_cast<float4 *>(doff[a] + i) = *reinterpret_cast<const float4 *>(soff[a] + i);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            *reinterpret_cast<float4 *>(du[a] + i) = *reinterpret_cast<const float4 *>(su[a] + i);
        if (dw && sw) *reinterpret_cast<float4 *>(dw + i) = *reinterpret_cast<const float4 *>(sw + i);
        if (did) {
            int4 v = make_int4(-1, -1, -1, -1);
            if (sid) {
                v = *reinterpret_cast<const int4 *>(sid + i);
                if (fill_dead) {  // (a dead slot keeps no id: its data is stale)
                    v.x = i < n_live ? v.x : -1;
                    v.y = i + 1 < n_live ? v.y : -1;
                    v.z = i + 2 < n_live ? v.z : -1;
                    v.w = i + 3 < n_live ? v.w : -1;
                }
            }
            *reinterpret_cast<int4 *>(did + i) = v;
        }
        return;
    }
    for (long long j = i; j < n; ++j) {
        dc[j] = (!fill_dead || j < n_live) ? sc[j] : -1;
#pragma unroll
        for (int a = 0; a < DIM; ++a) doff[a][j] = soff[a][j];
#pragma unroll
        for (int a = 0; a < 3; ++a) du[a][j] = su[a][j];
        if (dw && sw) dw[j] = sw[j];
        if (did) did[j] = sid && (!fill_dead || j < n_live) ? sid[j] : -1;
    }
}

template <int DIM>
__global__ void part_copy_kernel(const Run *__restrict__ run, PartCopy pc, long long n, int restore, FieldCopy fc)
{
    const Run &r = *run;
    const RunState &s = *r.state;
    const ParticleBuf pb = r.P[s.buf];
    const long long nq = (n + 3) / 4;
    // 16-byte accesses only if every buffer allows them
    uintptr_t al = (uintptr_t)pb.cell | (uintptr_t)pc.cell | (uintptr_t)pb.w | (uintptr_t)pc.w | (uintptr_t)pb.id |
                   (uintptr_t)pc.id;
#pragma unroll
    for (int a = 0; a < 3; ++a) al |= (uintptr_t)pb.u[a] | (uintptr_t)pc.u[a];
#pragma unroll
    for (int a = 0; a < DIM; ++a) al |= (uintptr_t)pb.off[a] | (uintptr_t)pc.off[a];
    const bool vec = (al & 15u) == 0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (long long)gridDim.x * blockDim.x) {
        if (!restore)
            copy4<DIM>(pc.cell, pc.off, pc.u, pc.w, pc.id, pb.cell, pb.off, pb.u, pb.w, pb.id, 4 * q, n, s.n_total,
                       true, vec);
        else
            copy4<DIM>(pb.cell, pb.off, pb.u, pb.w, pc.id ? pb.id : nullptr, pc.cell, pc.off, pc.u, pc.w, pc.id,
                       4 * q, n, 0, false, vec);
    }
    // fields and tile offsets of a record
    const long long nf = (long long)fc.nf * fc.cells;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nf + fc.nt;
         j += (long long)gridDim.x * blockDim.x) {
        if (j < nf) {
            const int c = (int)(j / fc.cells);
            const long long i = j - c * fc.cells;
            fc.dst[c][i] = fc.src[c][i];
        } else {
            fc.toff_dst[j - nf] = fc.toff_src[j - nf];
        }
    }
}

unsigned blocks_for(long long n)
{
    long long b = (n + kBlock - 1) / kBlock;
    return (unsigned)(b < 1 ? 1 : (b > 65535 * 4 ? 65535 * 4 : b));
}

}  // namespace

cudaError_t launch_adj_fields(int dim, const Run *run, AdjPtrs &A, int ncell, int plane, int origin, double t_n,
                              double dt, int laser_on, double *la0, cudaStream_t st)
{
    const unsigned g = blocks_for(ncell), gp = blocks_for(plane);
    if (dim == 2) {
        adj_b_kernel<2><<<g, kBlock, 0, st>>>(run, A, origin, t_n + dt, laser_on, la0, 1);
        adj_mur_kernel<2><<<gp, kBlock, 0, st>>>(run, A, origin);
        adj_e_curl_kernel<2><<<g, kBlock, 0, st>>>(run, A, origin, t_n, laser_on, la0);
    } else {
        adj_b_kernel<3><<<g, kBlock, 0, st>>>(run, A, origin, t_n + dt, laser_on, la0, 1);
        adj_mur_kernel<3><<<gp, kBlock, 0, st>>>(run, A, origin);
        adj_e_curl_kernel<3><<<g, kBlock, 0, st>>>(run, A, origin, t_n, laser_on, la0);
    }
    // lamE <- newE (the buffers trade places), then (iii)
    for (int c = 0; c < 3; ++c) std::swap(A.lE[c], A.nE[c]);
    if (dim == 2) adj_b_kernel<2><<<g, kBlock, 0, st>>>(run, A, origin, t_n, laser_on, la0, 0);
    else adj_b_kernel<3><<<g, kBlock, 0, st>>>(run, A, origin, t_n, laser_on, la0, 0);
    return cudaGetLastError();
}

template <int DIM, int P>
cudaError_t launch_adj_t(const Run *run, const Run &hr, const AdjPtrs &A, const TrajStep &ts, int origin,
                         cudaStream_t st)
{
    constexpr int kAdjBlock = 128;  // matches the kernels' launch bounds
    if (!ts.tile_off) {
        const unsigned g = (unsigned)((ts.n - ts.first + kAdjBlock - 1) / kAdjBlock);
        adj_particles_kernel<DIM, P><<<g, kAdjBlock, 0, st>>>(run, A, ts, origin);
        return cudaGetLastError();
    }
    size_t fv = 1, jv = 1;
    for (int a = 0; a < DIM; ++a) {
        const int T = 1 << hr.tlog[a];
        fv *= (size_t)(T + 2 * hr.drift + Reach<P>::GLO + Reach<P>::GHI);
        jv *= (size_t)(T + 2 * hr.drift + Reach<P>::DLO + Reach<P>::DHI);
    }
    const size_t smem = sizeof(float) * (6 * fv + 3 * jv);
    // the default 2D tile (16 x 16, drift 2) has its geometry compiled in
    const bool ct = DIM == 2 && hr.tlog[0] == 4 && hr.tlog[1] == 4 && hr.drift == 2;
    auto k = ct ? adj_particles_tiled_kernel<DIM, P, 16, 16, 1, 2> : adj_particles_tiled_kernel<DIM, P, 0, 0, 0, 0>;
    static size_t attr[2] = {0, 0};
    if (smem > attr[ct]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[ct] = smem;
    }
    // enough CTAs for about four waves of three CTAs per SM
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    int nsplit = (int)((4ll * 3 * sms + hr.ntiles - 1) / hr.ntiles);
    nsplit = nsplit < 1 ? 1 : (nsplit > 8 ? 8 : nsplit);
    k<<<(unsigned)((long long)hr.ntiles * nsplit), kAdjBlock, smem, st>>>(run, A, ts, origin, nsplit);
    return cudaGetLastError();
}

cudaError_t launch_adj_particles(int dim, int order, const Run *run, const Run &hr, const AdjPtrs &A,
                                 const TrajStep &ts, int origin, cudaStream_t st)
{
    if (ts.n <= ts.first) return cudaSuccess;
    if (dim == 2) {
        if (order == 1) return launch_adj_t<2, 1>(run, hr, A, ts, origin, st);
        if (order == 2) return launch_adj_t<2, 2>(run, hr, A, ts, origin, st);
        return launch_adj_t<2, 3>(run, hr, A, ts, origin, st);
    }
    if (order == 1) return launch_adj_t<3, 1>(run, hr, A, ts, origin, st);
    if (order == 2) return launch_adj_t<3, 2>(run, hr, A, ts, origin, st);
    return launch_adj_t<3, 3>(run, hr, A, ts, origin, st);
}

cudaError_t launch_objective(const Run *run, int origin, const ObjArgs &o, double *red, long long cap, int seed,
                             const AdjPtrs &A, cudaStream_t st)
{
    const unsigned g = blocks_for(cap) < 1024 ? blocks_for(cap) : 1024;
    if (!seed) {
        obj_reduce_kernel<<<g, kBlock, 0, st>>>(run, origin, o, red);
    } else {
        obj_seed_kernel<<<blocks_for(cap), kBlock, 0, st>>>(run, origin, o, red, A);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_perm(int dim, const AdjPtrs &A, const int32_t *id, long long n, long long nid, int to_slots,
                            cudaStream_t st)
{
    adj_perm_kernel<<<blocks_for(n), kBlock, 0, st>>>(A, id, n, nid, dim, to_slots);
    return cudaGetLastError();
}

cudaError_t launch_adj_window(const AdjPtrs &A, int plane, int store_plane, long long slot0, long long count,
                              long long id0, long long nid, cudaStream_t st)
{
    const long long m = plane > count ? plane : count;
    adj_window_kernel<<<blocks_for(m), kBlock, 0, st>>>(A, plane, store_plane, slot0, count, id0, nid);
    return cudaGetLastError();
}

cudaError_t launch_knots(const double *lw, const float *zb, long long n, int n_knots, double z0, double z1,
                         double ppc_t, double *out, cudaStream_t st)
{
    const unsigned g = blocks_for(n) < 608 ? blocks_for(n) : 608;
    knots_kernel<<<g, kBlock, 0, st>>>(lw, zb, n, n_knots, z0, z1, ppc_t, out);
    return cudaGetLastError();
}

cudaError_t launch_part_copy(int dim, const Run *run, const PartCopy &pc, long long n, int restore, cudaStream_t st)
{
    const long long nq = (n + 3) / 4;
    const FieldCopy none{};
    if (dim == 2) part_copy_kernel<2><<<blocks_for(nq), kBlock, 0, st>>>(run, pc, n, restore, none);
    else part_copy_kernel<3><<<blocks_for(nq), kBlock, 0, st>>>(run, pc, n, restore, none);
    return cudaGetLastError();
}

cudaError_t launch_record(int dim, const Run *run, const PartCopy &pc, long long n, const FieldCopy &fc,
                          cudaStream_t st)
{
    const long long nq = (n + 3) / 4;
    const long long work = nq > fc.nf * fc.cells + fc.nt ? nq : fc.nf * fc.cells + fc.nt;
    if (dim == 2) part_copy_kernel<2><<<blocks_for(work), kBlock, 0, st>>>(run, pc, n, 0, fc);
    else part_copy_kernel<3><<<blocks_for(work), kBlock, 0, st>>>(run, pc, n, 0, fc);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const Run *run, float *wid, float *zb, long long n, long long nid, cudaStream_t st)
{
    adj_init_kernel<<<blocks_for(n), kBlock, 0, st>>>(run, wid, zb, n, nid);
    return cudaGetLastError();
}

}  // namespace pic
