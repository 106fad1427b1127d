// Device code of the steady state-of-charge solver (sm_103a).
//
// One explicit pseudo-time sweep of Eq. nernst-planck-soc on a voxel lattice:
//   s'_c = s_c + dt * RHS_c,  RHS_c = adv_c + diff_c + k0 a_c R~(s_c)  (+ forcing)
// with first-order upwind advection by face velocities, 7-point diffusion, a Dirichlet
// inlet face and a zero-gradient outlet (Sec. III.C explicit operators), and the affine
// rate law R~(s) = A - B s (Eq. rate-from-soc-gen).
//
// Layout (structure of arrays, x fastest, c = i + nx*(j + ny*k)):
//   flags[c]  uint8: bit0 fluid, bits1..6 fluid neighbour at -x,+x,-y,+y,-z,+z,
//             bit7 electrode (fluid cell with at least one fiber neighbour)
//   u[c]      (beta/h) * velocity on the low-x face of cell c (0 for i = 0)
//   v[c]      (beta/h) * velocity on the low-y face
//   w[c]      (beta/h) * velocity on the low-z face; w[c + nx*ny] is the high face,
//             so w has N + nx*ny entries and its last plane holds the outlet faces.
// The high-x face of cell c is u[c+1] (zero at i = nx-1, a side wall), likewise y.
//
// Threads own one (i, j) column of a 32 x 8 tile and march a chunk of z planes,
// carrying s at k-1, k, k+1 and the shared z face in registers (2.5D streaming);
// x/y neighbours come through L1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rfb {

enum : unsigned {
    F_FLUID = 1u, F_XM = 2u, F_XP = 4u, F_YM = 8u, F_YP = 16u, F_ZM = 32u, F_ZP = 64u,
    F_ELEC = 128u
};
constexpr unsigned F_NBRS = 0x7Eu;

constexpr int BX = 32;
constexpr int BY = 8;
constexpr int NRED = 8;   // reduction slots of the FP64 check

struct Lattice {
    int nx, ny, nz, nxny;
    const uint8_t* __restrict__ flags;
    const uint8_t* __restrict__ mask32;   // mask byte of the FP32 kernels (below)
};

// Mask byte of the FP32 correction kernels: bit0 fluid, bit1 electrode, bits 2-4 the
// number of in-domain fluid neighbours n_f, bits 5-7 the number of fiber neighbours
// n_wall. These kernels keep the correction at 0 on solid and out-of-domain cells, so
// neighbour values need no per-face mask test: a solid or missing neighbour enters with
// value 0 and its face carries zero velocity.
constexpr unsigned M_FLUID = 1u, M_ELEC = 2u;
__device__ __forceinline__ int m_nf(unsigned m) { return (m >> 2) & 7u; }
__device__ __forceinline__ int m_nwall(unsigned m) { return m >> 5; }

template <typename T>
struct Coef {
    const T* __restrict__ u;
    const T* __restrict__ v;
    const T* __restrict__ w;
    const T* __restrict__ m;       // per-cell area multiplier, nullptr = 1
    const float* __restrict__ dtc; // per-cell step (local dt), nullptr = global dt
    T s_in;    // inlet value (0 in correction sweeps and U_mt)
    T Dh;      // D / h^2
    T gDh;     // inlet diffusion coefficient: 2 D/h^2 (face) or D/h^2 (ghost)
    T dt;      // global pseudo-time step
    T rA[8];   // k0 n_wall / h * A     by n_wall (zero in correction sweeps / U_mt);
               // kinetics mode 1: k0 n_wall / h * (e^{alpha eta~} - e^{(alpha-1) eta~})
    T rB[8];   // k0 n_wall / h * B     by n_wall (zero in U_mt); in mode 1 it only
               // bounds the pseudo-time step
    int umt;   // electrode cells are Dirichlet (value untouched), no reaction
    int nl;    // kinetics mode 1 (FP64 kernels only): source rA * g(s), see g_uniform
    T alpha;   // charge-transfer coefficient (mode 1)
};

// Kinetics mode 1, the Butler-Volmer rate at a uniform activation overpotential
// (Eq. source-term-bv-gen): R~(s) = K1 g(s) with g(s) = s^alpha (1-s)^(1-alpha) and
// K1 = e^{alpha eta~} - e^{(alpha-1) eta~}; g is evaluated on s clamped into [0, 1].
__device__ __forceinline__ double g_uniform(double s, double alpha) {
    s = fmin(fmax(s, 0.0), 1.0);
    if (alpha == 0.5) return sqrt(s * (1.0 - s));
    return pow(s, alpha) * pow(1.0 - s, 1.0 - alpha);
}

// g'(s) = s^(alpha-1) (1-s)^(-alpha) (alpha - s) = g(s) (alpha - s) / (s (1 - s)),
// for 0 < s < 1 (the adjoint's linearisation at a steady state).
__device__ __forceinline__ double g_uniform_slope(double s, double alpha) {
    return g_uniform(s, alpha) * (alpha - s) / (s * (1.0 - s));
}

// Source k0 a_c R~(s_c) of one cell from the per-n_wall tables: affine (A - B s), or
// mode 1 (FP64 only) K1 g(s).
template <typename T>
__device__ __forceinline__ T reaction(const Coef<T>& C, const T* tA, const T* tB, int nw,
                                      T mult, T sc) {
    if constexpr (sizeof(T) == 8) {
        if (C.nl) return mult * tA[nw] * g_uniform(sc, C.alpha);
    }
    return mult * (tA[nw] - tB[nw] * sc);
}

// q > 0 for an FP64 q, decided on the integer pipe (the FP64 pipe of GB300 is narrow);
// identical to the floating-point comparison for every non-NaN q, including -0.0.
__device__ __forceinline__ bool positive(double q) { return __double_as_longlong(q) > 0; }
__device__ __forceinline__ bool positive(float q) { return q > 0.0f; }

__device__ __forceinline__ int n_wall_of(unsigned f, int i, int j, int k, int nx, int ny,
                                         int nz) {
    int dom = 6 - (i == 0) - (i == nx - 1) - (j == 0) - (j == ny - 1) - (k == 0) -
              (k == nz - 1);
    return dom - __popc(f & F_NBRS);
}

// Right-hand side at one fluid cell. Neighbour values of non-fluid / out-of-domain
// neighbours must be passed as sc (their faces carry zero velocity and no diffusion).
// szm_adv: value carried in through the low-z face (s_in at the inlet).
// z_lo_dif: whether the low-z diffusion term is the inlet face term.
template <typename T>
__device__ __forceinline__ T cell_rhs(const Coef<T>& C, const T* tA, const T* tB, T sc, T sxm,
                                      T sxp, T sym, T syp, T szm, T szp, T uL, T uH, T vL,
                                      T vH, T wL, T wH, bool inlet, bool outlet, int nw,
                                      T mult) {
    // upwind advection: inflow through low faces, outflow through high faces
    T adv = uL * (positive(uL) ? sxm : sc);
    adv -= uH * (positive(uH) ? sc : sxp);
    adv += vL * (positive(vL) ? sym : sc);
    adv -= vH * (positive(vH) ? sc : syp);
    T zin = inlet ? C.s_in : szm;
    adv += wL * (positive(wL) ? zin : sc);
    T zout = outlet ? sc : szp;
    adv -= wH * (positive(wH) ? sc : zout);
    // 7-point diffusion between fluid cells (non-fluid neighbours enter as sc)
    T zmd = inlet ? sc : szm;
    T nsum = ((sxm + sxp) + (sym + syp)) + (zmd + szp);
    T dif = C.Dh * nsum - (T(6) * C.Dh) * sc;
    if (inlet) dif += C.gDh * (C.s_in - sc);
    // Butler-Volmer source k0 a_c R~(s)
    T rea = reaction<T>(C, tA, tB, nw, mult, sc);
    return (adv + dif) + rea;
}

// Diagonal d_c of -L at one fluid cell (outflow + diffusion + reaction), FP64.
template <typename T>
__device__ __forceinline__ T cell_diag(const Coef<T>& C, const T* tB, unsigned f, T uL, T uH,
                                       T vL, T vH, T wL, T wH, bool inlet, int nw, T mult) {
    T d = (uH > T(0) ? uH : T(0)) + (uL < T(0) ? -uL : T(0));
    d += (vH > T(0) ? vH : T(0)) + (vL < T(0) ? -vL : T(0));
    d += (wH > T(0) ? wH : T(0)) + (wL < T(0) ? -wL : T(0));
    d += C.Dh * T(__popc(f & F_NBRS));
    if (inlet) d += C.gDh;
    d += mult * tB[nw];
    return d;
}

// The per-n_wall reaction coefficients, copied once per block into shared memory
// (dynamic indexing of kernel-parameter arrays would go through local memory).
#define RFB_LOAD_TABLES(T, C)                                                         \
    __shared__ T tA[8], tB[8];                                                         \
    {                                                                                  \
        const int t_ = threadIdx.y * BX + threadIdx.x;                                 \
        if (t_ < 8) { tA[t_] = (C).rA[t_]; tB[t_] = (C).rB[t_]; }                      \
        __syncthreads();                                                               \
    }

// ---------------------------------------------------------------------------------
// Sweep: s_out = s + dt (RHS(s) [+ force]) on every unknown fluid cell. Cells that are
// solid (or pinned electrode cells in U_mt mode) are not written: both buffers hold
// the same fixed value there.
// ---------------------------------------------------------------------------------
template <typename T, bool FORCE>
__global__ void __launch_bounds__(BX * BY)
sweep_kernel(Lattice L, Coef<T> C, const T* __restrict__ s, T* __restrict__ s_out,
             const float* __restrict__ force, int kchunk) {
    RFB_LOAD_TABLES(T, C)
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= L.nx || j >= L.ny) return;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, L.nz);
    const int nx = L.nx, nxny = L.nxny;
    int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
    T s_prev = kb > 0 ? s[c - nxny] : T(0);
    T s_cur = s[c];
    T wL = C.w[c];
    for (int k = kb; k < ke; ++k, c += nxny) {
        const bool outlet = (k == L.nz - 1);
        T s_next = outlet ? T(0) : s[c + nxny];
        T wH = C.w[c + nxny];
        const unsigned f = L.flags[c];
        const bool upd = (f & F_FLUID) && !(C.umt && (f & F_ELEC));
        if (upd) {
            T sxm = (f & F_XM) ? s[c - 1] : s_cur;
            T sxp = (f & F_XP) ? s[c + 1] : s_cur;
            T sym = (f & F_YM) ? s[c - nx] : s_cur;
            T syp = (f & F_YP) ? s[c + nx] : s_cur;
            T szm = (f & F_ZM) ? s_prev : s_cur;
            T szp = (f & F_ZP) ? s_next : s_cur;
            T uL = C.u[c];
            T uH = (i + 1 < nx) ? C.u[c + 1] : T(0);
            T vL = C.v[c];
            T vH = (j + 1 < L.ny) ? C.v[c + nx] : T(0);
            const int nw = n_wall_of(f, i, j, k, nx, L.ny, L.nz);
            T mult = C.m ? C.m[c] : T(1);
            T r = cell_rhs<T>(C, tA, tB, s_cur, sxm, sxp, sym, syp, szm, szp, uL, uH, vL, vH, wL, wH,
                              k == 0, outlet, nw, mult);
            if (FORCE) r += T(force[c]);
            T dt = C.dtc ? T(C.dtc[c]) : C.dt;
            s_out[c] = s_cur + dt * r;
        }
        s_prev = s_cur;
        s_cur = s_next;
        wL = wH;
    }
}

// ---------------------------------------------------------------------------------
// FP32 correction sweep, vectorised: delta_out = delta + dt (L delta + r) with the
// homogeneous operator (no inlet value, no intercept), 4 consecutive x cells per thread
// (128-bit loads/stores, nx % 4 == 0). Every load of a plane is issued before any
// arithmetic (addresses are clamped at the domain edges instead of predicated on the
// flags), and the local step dt_c = cfl / d_c is computed on the fly from the FP32
// face velocities. Threads march a chunk of z planes keeping delta at k-1, k, k+1 and
// the shared z faces in registers.
// ---------------------------------------------------------------------------------
constexpr int VBX = 32;   // threads along x (128 cells)
constexpr int VBY = 8;

struct __align__(16) F4 { float x, y, z, w; };
__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float el(const float4& v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

template <bool LOCAL_DT, bool TR = false>
__global__ void __launch_bounds__(VBX * VBY)
sweep32v_kernel(Lattice L, Coef<float> C, const float* __restrict__ s,
                float* __restrict__ s_out, const float* __restrict__ force, float cfl,
                int kchunk);

// One FP32 correction update of one cell, delta' = delta + dt (L delta + r), with the
// homogeneous operator (zero inlet value, no intercept). The *_raw neighbour values are
// taken only where the flags say the neighbour is fluid (else the cell's own value), so
// out-of-domain or solid neighbours may hold anything finite. Shared by the plain and
// the temporally blocked sweeps, which therefore do bitwise the same arithmetic.
//
// The neighbour values must be 0 for solid and out-of-domain neighbours (the correction
// is 0 there and its boundary value at the inlet is 0): then every face term is right
// without testing the mask, since a face to a solid cell or a side wall has zero
// velocity, and the diffusion sum over all six neighbours equals the sum over fluid
// neighbours. The outlet face (zero gradient) is an outflow face (W >= 0 there), which
// the upwind choice already handles. rb = m_c k0 n_wall B / h, the reaction slope.
//
// In this form one update is linear in the seven values with coefficients fixed for the
// whole solve: s' = a_c s + sum_f a_f s_f + dt r, where a_f = dt (inflow through face f
// + D/h^2) and a_c = 1 - dt d_c with d_c = outflow + D/h^2 n_f (+ the inlet face term)
// + rb, the diagonal of -L. With the local step dt = cfl / d_c, a_c = 1 - cfl.
struct Coef32 {
    float a[6];   // -x, +x, -y, +y, -z, +z
    float ac;     // own value
    float dt;     // step (multiplies the forcing)
};

// The part of a cell's diagonal that depends only on its mask byte and on whether it
// lies on the inlet plane: D/h^2 n_f (+ the inlet face term) + rb, the reaction slope
// k0 m n_wall B / h; +inf for a cell that is not updated (solid, or a pinned electrode
// cell in U_mt mode).
__device__ __forceinline__ float dfix_of(unsigned m, bool inlet, int umt, float Dh, float gDh,
                                         float rb) {
    const bool upd = (m & M_FLUID) && !(umt && (m & M_ELEC));
    return upd ? fmaf(Dh, (float)m_nf(m), inlet ? gDh : 0.f) + rb : INFINITY;
}

// Per-block table of dfix_of for every mask byte (entries 0-255) and on the inlet plane
// (256-511), for lattices without area multipliers; tB: the block's copy of the
// per-n_wall reaction slopes. Callers synchronise the block before reading it.
constexpr int DFIX_TABLE = 512;
__device__ __forceinline__ void build_dfix_table(float* tdf, const float* tB, int umt, float Dh,
                                                 float gDh, int tid, int nthreads) {
    for (int q = tid; q < DFIX_TABLE; q += nthreads) {
        const unsigned m = (unsigned)q & 255u;
        tdf[q] = dfix_of(m, q >= 256, umt, Dh, gDh, tB[m_nwall(m)]);
    }
}

// Update coefficients of one cell: d = outflow + dfix is the diagonal of -L, the step is
// cfl / d (local) or the global one, a_f = dt (inflow_f + D/h^2) and a_c = 1 - dt d.
// TR: the same for the transposed operator L^T (adjoint), whose coefficient towards the
// neighbour across face f is that neighbour's inflow from this cell, i.e. this cell's
// outflow through f: a_f = dt (outflow_f + D/h^2); the diagonal is the same.
template <bool LOCAL_DT, bool TR = false>
__device__ __forceinline__ Coef32 cell_coef32(float dfix, float uL, float uH, float vL, float vH,
                                              float wl, float wh, float Dh, float cfl,
                                              float dt_global) {
    Coef32 k;
    const float d = (fmaxf(-uL, 0.f) + fmaxf(uH, 0.f)) + (fmaxf(-vL, 0.f) + fmaxf(vH, 0.f)) +
                    (fmaxf(-wl, 0.f) + fmaxf(wh, 0.f)) + dfix;
    const bool upd = dfix < INFINITY;
    float dt;
    if (LOCAL_DT) dt = (upd && d > 0.f) ? __fdividef(cfl, d) : 0.f;
    else dt = upd ? dt_global : 0.f;
    k.dt = dt;
    k.ac = dt > 0.f ? (LOCAL_DT ? 1.f - cfl : 1.f - dt * d) : 1.f;
    const float dtD = dt * Dh;
    const float sg = TR ? -1.f : 1.f;
    k.a[0] = fmaf(dt, fmaxf(sg * uL, 0.f), dtD);
    k.a[1] = fmaf(dt, fmaxf(-sg * uH, 0.f), dtD);
    k.a[2] = fmaf(dt, fmaxf(sg * vL, 0.f), dtD);
    k.a[3] = fmaf(dt, fmaxf(-sg * vH, 0.f), dtD);
    k.a[4] = fmaf(dt, fmaxf(sg * wl, 0.f), dtD);
    k.a[5] = fmaf(dt, fmaxf(-sg * wh, 0.f), dtD);
    return k;
}

// one update with the coefficients of cell_coef32 (cells that are not updated have
// dt = 0, a_f = 0, a_c = 1 and keep their value exactly)
__device__ __forceinline__ float cell_apply32(const Coef32& k, float sc, float xm, float xp,
                                              float ym, float yp, float zm, float zp, float r) {
    float acc = k.dt * r;
    acc = fmaf(k.a[0], xm, acc);
    acc = fmaf(k.a[1], xp, acc);
    acc = fmaf(k.a[2], ym, acc);
    acc = fmaf(k.a[3], yp, acc);
    acc = fmaf(k.a[4], zm, acc);
    acc = fmaf(k.a[5], zp, acc);
    return fmaf(k.ac, sc, acc);
}

// One tile of the vectorised sweep: columns (4 (bx VBX + tx) .. +3, by VBY + ty), planes
// kb .. ke-1. tB: the block's shared copy of the per-n_wall reaction slope.
template <bool LOCAL_DT, bool TR = false>
__device__ __forceinline__ void sweep32v_cells(const Lattice& L, const Coef<float>& C,
                                               const float* tB, const float* tdf,
                                               const float* __restrict__ s,
                                               float* __restrict__ s_out,
                                               const float* __restrict__ force, float cfl,
                                               int i0, int j, int kb, int ke);

template <bool LOCAL_DT, bool TR = false>
__device__ __forceinline__ void sweep32v_tile(const Lattice& L, const Coef<float>& C,
                                              const float* tB, const float* tdf,
                                              const float* __restrict__ s,
                                              float* __restrict__ s_out,
                                              const float* __restrict__ force, float cfl,
                                              int bx, int by, int kb, int ke) {
    const int i0 = 4 * (bx * VBX + threadIdx.x);
    const int j = by * VBY + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    sweep32v_cells<LOCAL_DT, TR>(L, C, tB, tdf, s, s_out, force, cfl, i0, j, kb, ke);
}

// The 4 cells (i0 .. i0+3, j) of every plane kb .. ke-1 (i0 % 4 == 0, nx % 4 == 0).
// tdf: the block's table of dfix_of (used when the lattice has no area multipliers).
// TR: a sweep of the transposed operator (adjoint correction).
template <bool LOCAL_DT, bool TR>
__device__ __forceinline__ void sweep32v_cells(const Lattice& L, const Coef<float>& C,
                                               const float* tB, const float* tdf,
                                               const float* __restrict__ s,
                                               float* __restrict__ s_out,
                                               const float* __restrict__ force, float cfl,
                                               int i0, int j, int kb, int ke) {
    const int nx = L.nx, ny = L.ny, nz = L.nz, nxny = L.nxny;
    const bool has_xm = i0 > 0, has_xp = i0 + 4 < nx;
    const bool has_ym = j > 0, has_yp = j + 1 < ny;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t c = (int64_t)i0 + (int64_t)nx * j + (int64_t)nxny * kb;
    float4 d_prev = kb > 0 ? ldg4(s + c - nxny) : zero4;   // plane -1: outside, 0
    float4 d_cur = ldg4(s + c);
    float4 wL = ldg4(C.w + c);
    const float Dh = C.Dh, gDh = C.gDh;
    for (int k = kb; k < ke; ++k, c += nxny) {
        const bool outlet = (k == nz - 1);
        const bool inlet = (k == 0);
        // ---- all loads of this plane (outside the domain the correction is 0)
        const float4 d_next = outlet ? zero4 : ldg4(s + c + nxny);
        const float4 wH = ldg4(C.w + c + nxny);
        const float4 d_ym = has_ym ? ldg4(s + c - nx) : zero4;
        const float4 d_yp = has_yp ? ldg4(s + c + nx) : zero4;
        const float d_xm = has_xm ? __ldg(s + c - 1) : 0.f;
        const float d_xp = has_xp ? __ldg(s + c + 4) : 0.f;
        const float4 u4 = ldg4(C.u + c);
        const float u_nx = has_xp ? __ldg(C.u + c + 4) : 0.f;
        const float4 v4 = ldg4(C.v + c);
        const float4 vH4 = has_yp ? ldg4(C.v + c + nx) : zero4;
        const float4 r4 = ldg4(force + c);
        const uint32_t m4b = __ldg(reinterpret_cast<const unsigned int*>(L.mask32 + c));
        const float4 m4 = C.m ? ldg4(C.m + c) : make_float4(1.f, 1.f, 1.f, 1.f);
        // ---- arithmetic
        float out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned m = (m4b >> (8 * e)) & 0xffu;
            const float dfix = C.m ? dfix_of(m, inlet, C.umt, Dh, gDh, el(m4, e) * tB[m_nwall(m)])
                                   : tdf[(inlet ? 256 : 0) + m];
            const Coef32 kc = cell_coef32<LOCAL_DT, TR>(
                dfix, el(u4, e), e == 3 ? u_nx : el(u4, e + 1), el(v4, e), el(vH4, e),
                el(wL, e), el(wH, e), Dh, cfl, C.dt);
            out[e] = cell_apply32(kc, el(d_cur, e), e == 0 ? d_xm : el(d_cur, e - 1),
                                  e == 3 ? d_xp : el(d_cur, e + 1), el(d_ym, e), el(d_yp, e),
                                  el(d_prev, e), el(d_next, e), el(r4, e));
        }
        *reinterpret_cast<float4*>(s_out + c) = make_float4(out[0], out[1], out[2], out[3]);
        d_prev = d_cur;
        d_cur = d_next;
        wL = wH;
    }
}

template <bool LOCAL_DT, bool TR>
__global__ void __launch_bounds__(VBX * VBY)
sweep32v_kernel(Lattice L, Coef<float> C, const float* __restrict__ s,
                float* __restrict__ s_out, const float* __restrict__ force, float cfl,
                int kchunk) {
    __shared__ float tB[8];
    __shared__ float tdf[DFIX_TABLE];
    {
        const int t_ = threadIdx.y * VBX + threadIdx.x;
        if (t_ < 8) tB[t_] = C.rB[t_];
        __syncthreads();
        build_dfix_table(tdf, tB, C.umt, C.Dh, C.gDh, t_, VBX * VBY);
        __syncthreads();
    }
    const int kb = blockIdx.z * kchunk;
    sweep32v_tile<LOCAL_DT, TR>(L, C, tB, tdf, s, s_out, force, cfl, blockIdx.x, blockIdx.y,
                                kb, min(kb + kchunk, L.nz));
}

// ---------------------------------------------------------------------------------
// Batches: many lattices of uneven size advanced by one persistent launch per sweep.
// Every lattice is cut into work items (1024 consecutive cells of the flattened x-y plane,
// 4 a thread, times a chunk of z planes); a grid of blocks walks the item list in a fixed
// round-robin order (the autotuner picks the grid size, from the resident blocks up to one
// block per item). Items of lattices that have converged are
// skipped (their `active` flag lives in device memory, so a captured CUDA graph keeps
// working as lattices drop out).
// ---------------------------------------------------------------------------------
// The assembled operator as double-float pairs (check_df_kernel below)
struct L2F {
    const float2* __restrict__ f[6];   // neighbour coefficients as (hi, lo)
    const float2* __restrict__ diag;
    const float2* __restrict__ b;
};

struct BatchInst {
    Lattice L;
    Coef<float> C32;       // correction sweep coefficients (homogeneous operator)
    Coef<double> C64;      // FP64 check coefficients (full operator)
    float* delta[2];
    float* r32;
    double* s64[2];
    L2F K2;                // double-float operator (double-float checks)
    float2* sdf[2];        // double-float state (double-float checks)
    float cfl;
    int active;            // 1 while the lattice has not converged
    int cur;               // which s64 (sdf with double-float checks) buffer holds the state
    int pad_;
};

struct BatchItem {
    int inst;
    int bx;        // first 4-cell group of the item in the flattened x-y plane (256 groups)
    int by;        // unused (0)
    int kb, ke;    // planes kb .. ke-1
};

template <bool LOCAL_DT>
__global__ void __launch_bounds__(VBX * VBY, 3)
batch_sweep_kernel(const BatchInst* __restrict__ insts, const BatchItem* __restrict__ items,
                   int n_items, int parity) {
    __shared__ float tB[8];
    __shared__ float tdf[DFIX_TABLE];
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const BatchItem it = items[w];
        const BatchInst* I = insts + it.inst;
        if (!I->active) continue;   // uniform over the block
        // copies in registers: read through the descriptor, every field would be reloaded
        // after each store (the compiler cannot rule out aliasing)
        const Lattice L = I->L;
        const Coef<float> C = I->C32;
        const float* src = I->delta[parity];
        float* dst = I->delta[parity ^ 1];
        const float* r32 = I->r32;
        const float cfl = I->cfl;
        __syncthreads();
        const int t = threadIdx.y * VBX + threadIdx.x;
        if (t < 8) tB[t] = I->C32.rB[t];
        __syncthreads();
        if (!C.m) {
            build_dfix_table(tdf, tB, C.umt, C.Dh, C.gDh, t, VBX * VBY);
            __syncthreads();
        }
        // the item covers 4-cell groups it.bx .. it.bx + 255 of the flattened x-y plane
        // (a group never crosses a row because nx % 4 == 0)
        const int64_t cell = 4 * ((int64_t)it.bx + t);
        if (cell < (int64_t)L.nxny)
            sweep32v_cells<LOCAL_DT>(L, C, tB, tdf, src, dst, r32, cfl, (int)(cell % L.nx),
                                     (int)(cell / L.nx), it.kb, it.ke);
    }
}

// delta := 0 on both buffers of every active lattice (start of a correction cycle)
__global__ void batch_zero_kernel(const BatchInst* __restrict__ insts, int n_inst) {
    for (int q = 0; q < n_inst; ++q) {
        const BatchInst& I = insts[q];
        if (!I.active) continue;
        const int64_t n = (int64_t)I.L.nxny * I.L.nz;
        float4* a = reinterpret_cast<float4*>(I.delta[0]);
        float4* b = reinterpret_cast<float4*>(I.delta[1]);
        for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n / 4;
             c += (int64_t)gridDim.x * blockDim.x) {
            a[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            b[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// ---------------------------------------------------------------------------------
// FP64 operator in coefficient form. For one operating point, RHS(s)_c =
//   b_c + L_cc s_c + sum_f L_f(c) s_f
// with L_f(c) = inflow through face f + D/h^2 (fluid neighbours only), L_cc = -(outflow +
// D/h^2 n_f + inlet face term + m k0 n_wall B / h) and b_c = inlet inflow and face terms
// times s_in + m k0 n_wall A / h. Assembled once per solve (FP64, 8 doubles a cell), it
// turns the FP64 sweep, check and adjoint into about 8 DFMAs a cell, which matters on
// GB300 whose FP64 rate is a small fraction of its FP32 rate. Rows of solid and pinned
// (U_mt) cells are all zero.
// ---------------------------------------------------------------------------------
struct L64 {
    double* __restrict__ f[6];   // neighbour coefficients: -x, +x, -y, +y, -z, +z
    double* __restrict__ diag;   // L_cc
    double* __restrict__ b;      // source
};

__device__ __forceinline__ void block_reduce_store(double (&acc)[NRED], double* out);

__global__ void assemble64_kernel(Lattice L, Coef<double> C, L64 K) {
    __shared__ double tA[8], tB[8];
    if (threadIdx.x < 8) { tA[threadIdx.x] = C.rA[threadIdx.x]; tB[threadIdx.x] = C.rB[threadIdx.x]; }
    __syncthreads();
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int64_t nxny = L.nxny, N = nxny * nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = L.flags[c];
        double a[6] = {0, 0, 0, 0, 0, 0}, dg = 0.0, bb = 0.0;
        if ((f & F_FLUID) && !(C.umt && (f & F_ELEC))) {
            const int i = (int)(c % nx);
            const int j = (int)((c / nx) % ny);
            const int k = (int)(c / nxny);
            const double uL = C.u[c], uH = (i + 1 < nx) ? C.u[c + 1] : 0.0;
            const double vL = C.v[c], vH = (j + 1 < ny) ? C.v[c + nx] : 0.0;
            const double wL = C.w[c], wH = C.w[c + nxny];
            const double Dh = C.Dh;
            // inflow coefficients (upwind) and diffusion to fluid neighbours
            a[0] = fmax(uL, 0.0) + ((f & F_XM) ? Dh : 0.0);
            a[1] = fmax(-uH, 0.0) + ((f & F_XP) ? Dh : 0.0);
            a[2] = fmax(vL, 0.0) + ((f & F_YM) ? Dh : 0.0);
            a[3] = fmax(-vH, 0.0) + ((f & F_YP) ? Dh : 0.0);
            a[4] = (k > 0) ? fmax(wL, 0.0) + ((f & F_ZM) ? Dh : 0.0) : 0.0;
            a[5] = fmax(-wH, 0.0) + ((f & F_ZP) ? Dh : 0.0);
            const double outflow = (fmax(-uL, 0.0) + fmax(uH, 0.0)) +
                                   (fmax(-vL, 0.0) + fmax(vH, 0.0)) +
                                   (fmax(-wL, 0.0) + fmax(wH, 0.0));
            const int nw = n_wall_of(f, i, j, k, nx, ny, nz);
            const double mult = C.m ? C.m[c] : 1.0;
            dg = -(outflow + Dh * (double)__popc(f & F_NBRS) + (k == 0 ? C.gDh : 0.0) +
                   mult * tB[nw]);
            bb = mult * tA[nw];
            if (k == 0) bb += (fmax(wL, 0.0) + C.gDh) * C.s_in;
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) K.f[q][c] = a[q];
        K.diag[c] = dg;
        K.b[c] = bb;
    }
}

// RHS at one cell from the assembled coefficients; neighbour values of missing
// neighbours may be anything finite (their coefficient is 0).
__device__ __forceinline__ double rhs64(const L64& K, int64_t c, double sc, double sxm, double sxp,
                                        double sym, double syp, double szm, double szp) {
    double r = fma(K.diag[c], sc, K.b[c]);
    r = fma(K.f[0][c], sxm, r);
    r = fma(K.f[1][c], sxp, r);
    r = fma(K.f[2][c], sym, r);
    r = fma(K.f[3][c], syp, r);
    r = fma(K.f[4][c], szm, r);
    r = fma(K.f[5][c], szp, r);
    return r;
}

// FP64 sweep s_out = s + dt RHS(s) with the assembled operator (2.5D z marching).
// NL (kinetics mode 1): the operator holds transport only; the source
// k_c g(s_c), k_c = m_c rA[n_wall], is added per cell; the step is capped by the source's
// local stiffness, dt <= cfl / (d_T + k_c max(0, -g'(s))) with d_T = -diag the transport
// diagonal and the slope taken at min(s, 1 - 2^-40) (near s = 1 it grows like
// (1-s)^(-alpha)); the update is clipped into [0, 1] (a guard that does not bind at a
// steady state). C and cfl are read only for NL.
template <bool NL>
__global__ void __launch_bounds__(BX * BY)
sweep64c_kernel(Lattice L, L64 K, const float* __restrict__ dtc, double dt_global,
                const double* __restrict__ s, double* __restrict__ s_out, int umt, int kchunk,
                Coef<double> C, double cfl) {
    __shared__ double tK[8];
    if (NL) {
        const int t = threadIdx.y * BX + threadIdx.x;
        if (t < 8) tK[t] = C.rA[t];
        __syncthreads();
    }
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= L.nx || j >= L.ny) return;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, L.nz);
    const int nx = L.nx, nxny = L.nxny;
    const int64_t oxm = i > 0 ? -1 : 0, oxp = i + 1 < nx ? 1 : 0;
    const int64_t oym = j > 0 ? -nx : 0, oyp = j + 1 < L.ny ? nx : 0;
    int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
    double s_prev = kb > 0 ? s[c - nxny] : 0.0;
    double s_cur = s[c];
    for (int k = kb; k < ke; ++k, c += nxny) {
        const double s_next = (k + 1 < L.nz) ? s[c + nxny] : 0.0;
        const unsigned f = L.flags[c];
        if ((f & F_FLUID) && !(umt && (f & F_ELEC))) {
            double r = rhs64(K, c, s_cur, s[c + oxm], s[c + oxp], s[c + oym], s[c + oyp],
                             s_prev, s_next);
            const double dt = dtc ? (double)dtc[c] : dt_global;
            if (NL) {
                const int nw = n_wall_of(f, i, j, k, nx, L.ny, L.nz);
                const double kc = (C.m ? C.m[c] : 1.0) * tK[nw];
                r += kc * g_uniform(s_cur, C.alpha);
                const double sh = fmin(s_cur, 1.0 - 0x1p-40);
                const double sl = (kc != 0.0 && sh > C.alpha) ? -g_uniform_slope(sh, C.alpha)
                                                              : 0.0;
                const double cap = cfl / (kc * sl - K.diag[c]);
                s_out[c] = fmin(fmax(fma(fmin(dt, cap), r, s_cur), 0.0), 1.0);
            } else {
                s_out[c] = fma(dt, r, s_cur);
            }
        }
        s_prev = s_cur;
        s_cur = s_next;
    }
}

// ---------------------------------------------------------------------------------
// Nernst model (Sec. II.D, Eqs. nernst-eta-inst-def,
// nernst-model-eta-update, nernst-model-s-update; Algorithm 8), FP64 on the assembled
// operator of the affine (SBV) problem. Electrode cells (k_c = m_c k0 n_wall / h > 0)
// hold s = sigma(V~ - eta~); their transport rate is T = RHS_SBV(s) - k_c (A - B s) (the
// operator without the cell's source), the instantaneous overpotential
//   eta~_I = 2 asinh(-T / (2 k_c sqrt(s (1 - s)))),
// and eta~ <- (1 - w) eta~ + w eta~_I with w = omega / (1 + |G|), G the slope of that map:
//   G = (-d_T sqrt(s(1-s)) / k_c + (1 - 2 s) sinh(eta~/2)) / cosh(eta~/2),
// d_T = the transport diagonal (one weight for all cells would have to stay below
// 2 / (1 + |G|) everywhere); G is evaluated in FP32 (GB300's FP64 transcendentals are
// slow). Other unknown cells take the explicit step s + dt RHS.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double sigmoid64(double x) { return 1.0 / (1.0 + exp(-x)); }

// k0 a_c of fluid cell c (0 on cells without fiber neighbours or with multiplier 0)
__device__ __forceinline__ double nernst_kc(const Lattice& L, const Coef<double>& C, int64_t c,
                                            unsigned f, double kap0) {
    const int i = (int)(c % L.nx);
    const int j = (int)((c / L.nx) % L.ny);
    const int k = (int)(c / L.nxny);
    return (C.m ? C.m[c] : 1.0) * kap0 * n_wall_of(f, i, j, k, L.nx, L.ny, L.nz);
}

// The electrode cells as a list (warp-aggregated appends: each warp's cells stay
// together and in order; which warp comes first does not matter, every cell's update is
// independent of the others within a step).
__global__ void nernst_list_kernel(Lattice L, Coef<double> C, double kap0,
                                   int* __restrict__ list, int* __restrict__ count) {
    const int64_t N = (int64_t)L.nxny * L.nz;
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < N;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = base + threadIdx.x;
        bool e = false;
        if (c < N) {
            const unsigned f = L.flags[c];
            e = (f & F_FLUID) && nernst_kc(L, C, c, f, kap0) > 0.0;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, e);
        int first = 0;
        if (lane == 0 && mask) first = atomicAdd(count, __popc(mask));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (e) list[first + __popc(mask & ((1u << lane) - 1u))] = (int)c;
    }
}

// Interior step: s_out = s + dt RHS(s) on unknown cells that are not electrode cells.
__global__ void __launch_bounds__(BX * BY)
nernst_interior_kernel(Lattice L, L64 K, Coef<double> C, const float* __restrict__ dtc,
                       double dt_global, const double* __restrict__ s,
                       double* __restrict__ s_out, double kap0, int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= L.nx || j >= L.ny) return;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, L.nz);
    const int nx = L.nx, nxny = L.nxny;
    const int64_t oxm = i > 0 ? -1 : 0, oxp = i + 1 < nx ? 1 : 0;
    const int64_t oym = j > 0 ? -nx : 0, oyp = j + 1 < L.ny ? nx : 0;
    int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
    double s_prev = kb > 0 ? s[c - nxny] : 0.0;
    double s_cur = s[c];
    for (int k = kb; k < ke; ++k, c += nxny) {
        const double s_next = (k + 1 < L.nz) ? s[c + nxny] : 0.0;
        const unsigned f = L.flags[c];
        const bool elec = (f & F_ELEC) && (!C.m || C.m[c] > 0.0) && kap0 > 0.0;
        if ((f & F_FLUID) && !elec) {
            const double r = rhs64(K, c, s_cur, s[c + oxm], s[c + oxp], s[c + oym], s[c + oyp],
                                   s_prev, s_next);
            const double dt = dtc ? (double)dtc[c] : dt_global;
            s_out[c] = fma(dt, r, s_cur);
        }
        s_prev = s_cur;
        s_cur = s_next;
    }
}

// Electrode step over the list: T = RHS_SBV(s) - k_c (A - B s), eta~_I, the relaxed
// eta~ update and s_out = sigma(V~ - eta~).
__global__ void nernst_elec_kernel(Lattice L, L64 K, Coef<double> C,
                                   const int* __restrict__ list, int n,
                                   const double* __restrict__ s, double* __restrict__ s_out,
                                   double* __restrict__ eta_t, double kap0, double Vt,
                                   double omega) {
    __shared__ double tA[8], tB[8];
    if (threadIdx.x < 8) { tA[threadIdx.x] = C.rA[threadIdx.x]; tB[threadIdx.x] = C.rB[threadIdx.x]; }
    __syncthreads();
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int64_t nxny = L.nxny;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int64_t c = list[q];
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / nxny);
        const double sc0 = s[c];
        const double r = rhs64(K, c, sc0, s[c - (i > 0)], s[c + (i + 1 < nx)],
                               s[c - (j > 0 ? nx : 0)], s[c + (j + 1 < ny ? nx : 0)],
                               s[c - (k > 0 ? nxny : 0)], s[c + (k + 1 < nz ? nxny : 0)]);
        const unsigned f = L.flags[c];
        const int nw = n_wall_of(f, i, j, k, nx, ny, nz);
        const double mult = C.m ? C.m[c] : 1.0;
        const double kc = mult * kap0 * nw;
        const double T = r - mult * (tA[nw] - tB[nw] * sc0);
        const double dT = -K.diag[c] - mult * tB[nw];
        const double sc = fmin(fmax(sc0, 1e-300), 1.0 - 0x1p-53);
        const double root = sqrt(sc * (1.0 - sc));
        const double e = eta_t[c];
        const double ei = 2.0 * asinh(-T / (2.0 * kc * root));
        // the relaxation weight only sets the step (the fixed point does not depend on
        // it): FP32, one exponential for sinh and cosh
        const float ex = __expf(0.5f * (float)e), exi = 1.0f / ex;
        const float G = (-(float)(dT / kc) * (float)root +
                         (float)(1.0 - 2.0 * sc) * 0.5f * (ex - exi)) / (0.5f * (ex + exi));
        const double w = omega / (1.0 + (double)fabsf(G));
        const double en = fma(w, ei - e, e);
        eta_t[c] = en;
        s_out[c] = sigmoid64(Vt - en);
    }
}

// Start of a Nernst solve: eta~ = 0 and s = sigma(V~) on electrode cells (cold), or
// eta~ = V~ - logit(s) from the current state (warm); 0 off the electrode cells.
__global__ void nernst_init_kernel(Lattice L, Coef<double> C, double* __restrict__ sa,
                                   double* __restrict__ sb, double* __restrict__ eta_t,
                                   double kap0, double Vt, int warm) {
    const int64_t N = (int64_t)L.nxny * L.nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = L.flags[c];
        double e = 0.0;
        if (f & F_FLUID) {
            const int i = (int)(c % L.nx);
            const int j = (int)((c / L.nx) % L.ny);
            const int k = (int)(c / L.nxny);
            const int nw = n_wall_of(f, i, j, k, L.nx, L.ny, L.nz);
            const double kc = (C.m ? C.m[c] : 1.0) * kap0 * nw;
            if (kc > 0.0) {
                if (warm) {
                    const double s = fmin(fmax(sa[c], 1e-300), 1.0 - 0x1p-53);
                    e = Vt - log(s / (1.0 - s));
                } else {
                    sa[c] = sb[c] = sigmoid64(Vt);
                }
            }
        }
        eta_t[c] = e;
    }
}

// Kinetics mode 1: adds the source's derivative m_c rA[n_wall] g'(s_c) to the assembled
// diagonal, so that the operator becomes the Jacobian dRHS/ds at the state s (the
// adjoint of the nonlinear steady state).
__global__ void linearise64_kernel(Lattice L, Coef<double> C, L64 K,
                                   const double* __restrict__ s) {
    __shared__ double tK[8];
    if (threadIdx.x < 8) tK[threadIdx.x] = C.rA[threadIdx.x];
    __syncthreads();
    const int64_t N = (int64_t)L.nxny * L.nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = L.flags[c];
        if (!(f & F_FLUID) || (C.umt && (f & F_ELEC))) continue;
        const int i = (int)(c % L.nx);
        const int j = (int)((c / L.nx) % L.ny);
        const int k = (int)(c / L.nxny);
        const int nw = n_wall_of(f, i, j, k, L.nx, L.ny, L.nz);
        if (nw == 0) continue;
        const double mult = C.m ? C.m[c] : 1.0;
        K.diag[c] += mult * tK[nw] * g_uniform_slope(s[c], C.alpha);
    }
}

// Transposed step with the assembled operator: (L^T lam)_c gathers, from each neighbour
// row, the coefficient that points back to c (e.g. from the +x neighbour its -x
// coefficient). MODE 0: lam_out = lam + dt (L^T lam + g); MODE 1: reductions of
// r = L^T lam + g over unknown cells (0 sum r^2, 1 sum g^2, 6 non-finite, 7 max |r|).
template <int MODE>
__global__ void __launch_bounds__(BX * BY)
adjoint64c_kernel(Lattice L, L64 K, const float* __restrict__ dtc, double dt_global,
                  const double* __restrict__ lam, double* __restrict__ lam_out,
                  const double* __restrict__ g, double* __restrict__ partials, int umt,
                  int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    if (i < L.nx && j < L.ny) {
        const int kb = blockIdx.z * kchunk;
        const int ke = min(kb + kchunk, L.nz);
        const int nx = L.nx, ny = L.ny, nz = L.nz, nxny = L.nxny;
        int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
        double l_prev = kb > 0 ? lam[c - nxny] : 0.0;
        double l_cur = lam[c];
        for (int k = kb; k < ke; ++k, c += nxny) {
            const double l_next = (k + 1 < nz) ? lam[c + nxny] : 0.0;
            const unsigned f = L.flags[c];
            if ((f & F_FLUID) && !(umt && (f & F_ELEC))) {
                double r = fma(K.diag[c], l_cur, g[c]);
                if (i > 0) r = fma(K.f[1][c - 1], lam[c - 1], r);
                if (i + 1 < nx) r = fma(K.f[0][c + 1], lam[c + 1], r);
                if (j > 0) r = fma(K.f[3][c - nx], lam[c - nx], r);
                if (j + 1 < ny) r = fma(K.f[2][c + nx], lam[c + nx], r);
                if (k > 0) r = fma(K.f[5][c - nxny], l_prev, r);
                if (k + 1 < nz) r = fma(K.f[4][c + nxny], l_next, r);
                if (MODE == 0) {
                    const double dt = dtc ? (double)dtc[c] : dt_global;
                    lam_out[c] = fma(dt, r, l_cur);
                } else {
                    if (isfinite(r)) {
                        acc[0] += r * r;
                        acc[7] = fmax(acc[7], fabs(r));
                    } else {
                        acc[6] += 1.0;
                    }
                    acc[1] += g[c] * g[c];
                }
            }
            l_prev = l_cur;
            l_cur = l_next;
        }
    }
    if (MODE == 1) {
        const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                            ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
        block_reduce_store(acc, partials + bid * NRED);
    }
}

// ---------------------------------------------------------------------------------
// Block reduction helpers (fixed order => deterministic)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_max(double x) {
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    return x;
}

// slots 0..NRED-2 are sums, slot NRED-1 is a max
__device__ __forceinline__ void block_reduce_store(double (&acc)[NRED], double* out) {
    __shared__ double sh[BX * BY / 32][NRED];
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < NRED - 1; ++q) acc[q] = warp_sum(acc[q]);
    acc[NRED - 1] = warp_max(acc[NRED - 1]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NRED; ++q) sh[wid][q] = acc[q];
    }
    __syncthreads();
    if (tid < NRED) {
        double r = sh[0][tid];
        for (int w = 1; w < BX * BY / 32; ++w)
            r = (tid == NRED - 1) ? fmax(r, sh[w][tid]) : r + sh[w][tid];
        out[tid] = r;
    }
}

// ---------------------------------------------------------------------------------
// FP64 check: RHS64 at every fluid cell and the reductions
//   0 sum RHS^2 (unknown cells)        4 sum_outlet wH s
//   1 sum m kappa R~(s) (fluid cells)  5 sum_outlet wH
//   2 sum_inlet gDh (s_in - s)         6 count of non-finite RHS
//   3 sum_inlet wL s_in                7 max |RHS|
// FUSE: the state is s_old + delta (FP32 correction); it is written to s_new.
// WRITE_R: RHS is stored as FP32 forcing for the next correction sweeps.
// ---------------------------------------------------------------------------------
template <bool FUSE, bool WRITE_R>
__device__ __forceinline__ void check_column(const Lattice& L, const Coef<double>& C,
                                             const double* tA, const double* tB,
                                             const double* __restrict__ s,
                                             const float* __restrict__ delta,
                                             double* __restrict__ s_new,
                                             float* __restrict__ r_out, double (&acc)[NRED],
                                             int i, int j, int kb, int ke);

template <bool FUSE, bool WRITE_R>
__device__ __forceinline__ void check_tile(const Lattice& L, const Coef<double>& C,
                                           const double* tA, const double* tB,
                                           const double* __restrict__ s,
                                           const float* __restrict__ delta,
                                           double* __restrict__ s_new,
                                           float* __restrict__ r_out, double (&acc)[NRED],
                                           int bx, int by, int kb, int ke) {
    check_column<FUSE, WRITE_R>(L, C, tA, tB, s, delta, s_new, r_out, acc,
                                bx * BX + threadIdx.x, by * BY + threadIdx.y, kb, ke);
}

// FP64 RHS and reductions down the column (i, j), planes kb .. ke-1.
template <bool FUSE, bool WRITE_R>
__device__ __forceinline__ void check_column(const Lattice& L, const Coef<double>& C,
                                             const double* tA, const double* tB,
                                             const double* __restrict__ s,
                                             const float* __restrict__ delta,
                                             double* __restrict__ s_new,
                                             float* __restrict__ r_out, double (&acc)[NRED],
                                             int i, int j, int kb, int ke) {
    if (i < L.nx && j < L.ny) {
        const int nx = L.nx, nxny = L.nxny;
        auto val = [&](int64_t cc) -> double {
            return FUSE ? s[cc] + (double)delta[cc] : s[cc];
        };
        int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
        double s_prev = kb > 0 ? val(c - nxny) : 0.0;
        double s_cur = val(c);
        double wL = C.w[c];
        for (int k = kb; k < ke; ++k, c += nxny) {
            const bool outlet = (k == L.nz - 1);
            double s_next = outlet ? 0.0 : val(c + nxny);
            double wH = C.w[c + nxny];
            const unsigned f = L.flags[c];
            if (FUSE) s_new[c] = s_cur;
            if (f & F_FLUID) {
                const bool pinned = C.umt && (f & F_ELEC);
                double sxm = (f & F_XM) ? val(c - 1) : s_cur;
                double sxp = (f & F_XP) ? val(c + 1) : s_cur;
                double sym = (f & F_YM) ? val(c - nx) : s_cur;
                double syp = (f & F_YP) ? val(c + nx) : s_cur;
                double szm = (f & F_ZM) ? s_prev : s_cur;
                double szp = (f & F_ZP) ? s_next : s_cur;
                double uL = C.u[c];
                double uH = (i + 1 < nx) ? C.u[c + 1] : 0.0;
                double vL = C.v[c];
                double vH = (j + 1 < L.ny) ? C.v[c + nx] : 0.0;
                const int nw = n_wall_of(f, i, j, k, nx, L.ny, L.nz);
                double mult = C.m ? C.m[c] : 1.0;
                double r = cell_rhs<double>(C, tA, tB, s_cur, sxm, sxp, sym, syp, szm, szp, uL, uH,
                                            vL, vH, wL, wH, k == 0, outlet, nw, mult);
                if (!pinned) {
                    if (isfinite(r)) {
                        acc[0] += r * r;
                        acc[7] = fmax(acc[7], fabs(r));
                    } else {
                        acc[6] += 1.0;
                    }
                    if (WRITE_R) r_out[c] = (float)r;
                } else if (WRITE_R) {
                    r_out[c] = 0.0f;
                }
                acc[1] += reaction<double>(C, tA, tB, nw, mult, s_cur);
                if (k == 0) {
                    acc[2] += C.gDh * (C.s_in - s_cur);
                    acc[3] += wL * C.s_in;
                }
                if (outlet) {
                    acc[4] += wH * s_cur;
                    acc[5] += wH;
                }
            }
            s_prev = s_cur;
            s_cur = s_next;
            wL = wH;
        }
    }
}

template <bool FUSE, bool WRITE_R>
__global__ void __launch_bounds__(BX * BY)
check_kernel(Lattice L, Coef<double> C, const double* __restrict__ s,
             const float* __restrict__ delta, double* __restrict__ s_new,
             float* __restrict__ r_out, double* __restrict__ partials, int kchunk) {
    RFB_LOAD_TABLES(double, C)
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    const int kb = blockIdx.z * kchunk;
    check_tile<FUSE, WRITE_R>(L, C, tA, tB, s, delta, s_new, r_out, acc, blockIdx.x,
                              blockIdx.y, kb, min(kb + kchunk, L.nz));
    const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                        ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_reduce_store(acc, partials + bid * NRED);
}

// FP64 check with the assembled operator (same reductions and fusion as check_kernel);
// velocities are read only on the inlet and outlet planes, for the currents.
template <bool FUSE, bool WRITE_R>
__global__ void __launch_bounds__(BX * BY)
check64c_kernel(Lattice L, Coef<double> C, L64 K, const double* __restrict__ s,
                const float* __restrict__ delta, double* __restrict__ s_new,
                float* __restrict__ r_out, double* __restrict__ partials, int kchunk) {
    RFB_LOAD_TABLES(double, C)
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i < L.nx && j < L.ny) {
        const int kb = blockIdx.z * kchunk;
        const int ke = min(kb + kchunk, L.nz);
        const int nx = L.nx, nxny = L.nxny;
        const int64_t oxm = i > 0 ? -1 : 0, oxp = i + 1 < nx ? 1 : 0;
        const int64_t oym = j > 0 ? -nx : 0, oyp = j + 1 < L.ny ? nx : 0;
        auto val = [&](int64_t cc) -> double {
            return FUSE ? s[cc] + (double)delta[cc] : s[cc];
        };
        int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
        double s_prev = kb > 0 ? val(c - nxny) : 0.0;
        double s_cur = val(c);
        for (int k = kb; k < ke; ++k, c += nxny) {
            const bool outlet = (k == L.nz - 1);
            const double s_next = outlet ? 0.0 : val(c + nxny);
            const unsigned f = L.flags[c];
            if (FUSE) s_new[c] = s_cur;
            if (f & F_FLUID) {
                const bool pinned = C.umt && (f & F_ELEC);
                const int nw = n_wall_of(f, i, j, k, nx, L.ny, L.nz);
                const double mult = C.m ? C.m[c] : 1.0;
                const double src = reaction<double>(C, tA, tB, nw, mult, s_cur);
                if (!pinned) {
                    double r = rhs64(K, c, s_cur, val(c + oxm), val(c + oxp), val(c + oym),
                                     val(c + oyp), s_prev, s_next);
                    if (C.nl) r += src;   // mode 1: the operator holds transport only
                    if (isfinite(r)) {
                        acc[0] += r * r;
                        acc[7] = fmax(acc[7], fabs(r));
                    } else {
                        acc[6] += 1.0;
                    }
                    if (WRITE_R) r_out[c] = (float)r;
                } else if (WRITE_R) {
                    r_out[c] = 0.0f;
                }
                acc[1] += src;
                if (k == 0) {
                    acc[2] += C.gDh * (C.s_in - s_cur);
                    acc[3] += C.w[c] * C.s_in;
                }
                if (outlet) {
                    const double wH = C.w[c + nxny];
                    acc[4] += wH * s_cur;
                    acc[5] += wH;
                }
            }
            s_prev = s_cur;
            s_cur = s_next;
        }
    }
    const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                        ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_reduce_store(acc, partials + bid * NRED);
}

// ---------------------------------------------------------------------------------
// Mixed-precision defect check in double-float arithmetic. GB300 issues FP64 at a small
// fraction of its FP32 rate, and the FP64 check (about 25 FP64 operations a cell) runs
// several times longer than its HBM traffic takes. Here the assembled operator and the
// state are unevaluated sums hi + lo of two FP32 numbers (about 48 significant bits), and
// the defect is formed with error-free transformations on the FP32 pipes: Knuth's
// TwoSum, Dekker's FastTwoSum and the exact product through an FMA. The absolute error of
// a defect is about 2^-47 of its largest term, far below the tolerances of a solve; the
// last check of every mixed solve is the FP64 one.
// ---------------------------------------------------------------------------------

__device__ __forceinline__ float2 two_sum(float a, float b) {      // a + b = s + e exactly
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) { // needs |a| >= |b|
    const float s = a + b;
    return make_float2(s, b - (s - a));
}
// acc + a x for pairs: exact product of the high parts, the cross terms through FMAs
__device__ __forceinline__ float2 df_fma(float2 a, float2 x, float2 acc) {
    const float ph = a.x * x.x;
    float pl = fmaf(a.x, x.x, -ph);
    pl = fmaf(a.x, x.y, pl);
    pl = fmaf(a.y, x.x, pl);
    const float2 s = two_sum(acc.x, ph);
    return fast_two_sum(s.x, s.y + (acc.y + pl));
}
// pair + FP32 number
__device__ __forceinline__ float2 df_add_f(float2 a, float b) {
    const float2 s = two_sum(a.x, b);
    return fast_two_sum(s.x, s.y + a.y);
}

// pairs (hi, lo) of FP64 numbers: hi = rn(x), lo = rn(x - hi)
__global__ void split64_kernel(const double* __restrict__ in, float2* __restrict__ out, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double x = in[q];
        const float hi = __double2float_rn(x);
        out[q] = make_float2(hi, __double2float_rn(x - (double)hi));
    }
}
__global__ void join64_kernel(const float2* __restrict__ in, double* __restrict__ out, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = in[q];
        out[q] = (double)v.x + (double)v.y;
    }
}

// (Latency bound: four blocks per SM and the z-march unrolled by two keep more loads in
// flight.)
// The defect RHS(s [+ delta]) = b + L (s [+ delta]) at every unknown cell, written as the
// FP32 forcing (its high part), with the reductions the iteration needs: 0 sum RHS^2,
// 6 count of non-finite values, 7 max |RHS| (slots 1-5 stay 0). FUSE: the state is
// s + delta, written to s_new (every cell).
// One column (i, j), planes kb .. ke-1, of the double-float defect; accumulates the sum of
// squares, the largest magnitude and the non-finite count over unknown cells.
template <bool FUSE>
__device__ __forceinline__ void check_df_column(const Lattice& L, const L2F& K,
                                                const float2* __restrict__ s,
                                                const float* __restrict__ delta,
                                                float2* __restrict__ s_new,
                                                float* __restrict__ r_out, int umt, int i,
                                                int j, int kb, int ke, float& sum2, float& vmax,
                                                int& bad) {
    const int nx = L.nx, nxny = L.nxny;
    const int64_t oxm = i > 0 ? -1 : 0, oxp = i + 1 < nx ? 1 : 0;
    const int64_t oym = j > 0 ? -nx : 0, oyp = j + 1 < L.ny ? nx : 0;
    auto val = [&](int64_t cc) -> float2 {
        return FUSE ? df_add_f(s[cc], delta[cc]) : s[cc];
    };
    const float2 zero = make_float2(0.f, 0.f);
    int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
    float2 s_prev = kb > 0 ? val(c - nxny) : zero;
    float2 s_cur = val(c);
#pragma unroll 2
    for (int k = kb; k < ke; ++k, c += nxny) {
        const float2 s_next = (k + 1 < L.nz) ? val(c + nxny) : zero;
        const unsigned f = L.flags[c];
        if (FUSE) s_new[c] = s_cur;
        if (f & F_FLUID) {
            if (!(umt && (f & F_ELEC))) {
                float2 r = df_fma(K.diag[c], s_cur, K.b[c]);
                r = df_fma(K.f[0][c], val(c + oxm), r);
                r = df_fma(K.f[1][c], val(c + oxp), r);
                r = df_fma(K.f[2][c], val(c + oym), r);
                r = df_fma(K.f[3][c], val(c + oyp), r);
                r = df_fma(K.f[4][c], s_prev, r);
                r = df_fma(K.f[5][c], s_next, r);
                r_out[c] = r.x;
                const float q = r.x * r.x;
                if (isfinite(q)) {
                    sum2 += q;
                    vmax = fmaxf(vmax, fabsf(r.x));
                } else {
                    ++bad;
                }
            } else {
                r_out[c] = 0.f;
            }
        }
        s_prev = s_cur;
        s_cur = s_next;
    }
}

// Defect r = b + L s in double-float (s [+ delta] as pairs), written as the FP32 forcing;
// reductions 0 sum r^2, 6 non-finite count, 7 max |r| over unknown cells. FUSE: s + delta
// is the state, written to s_new (every cell).
template <bool FUSE>
__global__ void __launch_bounds__(BX * BY, 4)
check_df_kernel(Lattice L, L2F K, const float2* __restrict__ s, const float* __restrict__ delta,
                float2* __restrict__ s_new, float* __restrict__ r_out,
                double* __restrict__ partials, int umt, int kchunk) {
    float sum2 = 0.f, vmax = 0.f;
    int bad = 0;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i < L.nx && j < L.ny) {
        const int kb = blockIdx.z * kchunk;
        check_df_column<FUSE>(L, K, s, delta, s_new, r_out, umt, i, j, kb,
                              min(kb + kchunk, L.nz), sum2, vmax, bad);
    }
    double acc[NRED] = {(double)sum2, 0.0, 0.0, 0.0, 0.0, 0.0, (double)bad, (double)vmax};
    const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                        ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_reduce_store(acc, partials + bid * NRED);
}

// Adjoint defect r = g + L^T lam in double-float (lam [+ delta] as pairs): (L^T lam)_c
// gathers from each neighbour row the coefficient that points back to c. Written as the
// FP32 forcing; reductions 0 sum r^2, 1 sum g^2, 6 non-finite count, 7 max |r| over unknown
// cells. FUSE: lam + delta is the state, written to lam_new (every cell).
template <bool FUSE>
__global__ void __launch_bounds__(BX * BY, 4)
check_df_adjoint_kernel(Lattice L, L2F K, const float2* __restrict__ lam,
                        const float* __restrict__ delta, float2* __restrict__ lam_new,
                        const float2* __restrict__ g, float* __restrict__ r_out,
                        double* __restrict__ partials, int umt, int kchunk) {
    float sum2 = 0.f, sumg = 0.f, vmax = 0.f;
    int bad = 0;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i < L.nx && j < L.ny) {
        const int kb = blockIdx.z * kchunk;
        const int ke = min(kb + kchunk, L.nz);
        const int nx = L.nx, ny = L.ny, nz = L.nz, nxny = L.nxny;
        auto val = [&](int64_t cc) -> float2 {
            return FUSE ? df_add_f(lam[cc], delta[cc]) : lam[cc];
        };
        const float2 zero = make_float2(0.f, 0.f);
        int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
        float2 l_prev = kb > 0 ? val(c - nxny) : zero;
        float2 l_cur = val(c);
#pragma unroll 2
        for (int k = kb; k < ke; ++k, c += nxny) {
            const float2 l_next = (k + 1 < nz) ? val(c + nxny) : zero;
            const unsigned f = L.flags[c];
            if (FUSE) lam_new[c] = l_cur;
            if (f & F_FLUID) {
                if (!(umt && (f & F_ELEC))) {
                    const float2 gc = g[c];
                    float2 r = df_fma(K.diag[c], l_cur, gc);
                    if (i > 0) r = df_fma(K.f[1][c - 1], val(c - 1), r);
                    if (i + 1 < nx) r = df_fma(K.f[0][c + 1], val(c + 1), r);
                    if (j > 0) r = df_fma(K.f[3][c - nx], val(c - nx), r);
                    if (j + 1 < ny) r = df_fma(K.f[2][c + nx], val(c + nx), r);
                    if (k > 0) r = df_fma(K.f[5][c - nxny], l_prev, r);
                    if (k + 1 < nz) r = df_fma(K.f[4][c + nxny], l_next, r);
                    r_out[c] = r.x;
                    const float q = r.x * r.x;
                    if (isfinite(q)) {
                        sum2 += q;
                        vmax = fmaxf(vmax, fabsf(r.x));
                    } else {
                        ++bad;
                    }
                    sumg += gc.x * gc.x;
                } else {
                    r_out[c] = 0.f;
                }
            }
            l_prev = l_cur;
            l_cur = l_next;
        }
    }
    double acc[NRED] = {(double)sum2, (double)sumg, 0.0, 0.0, 0.0, 0.0, (double)bad,
                        (double)vmax};
    const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                        ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_reduce_store(acc, partials + bid * NRED);
}

// Batched FP64 check (FUSE: state = s64[cur] + delta[0] written to s64[cur ^ 1], FP32
// forcing refreshed), one work item per loop trip; partial sums per item. Items of
// inactive lattices write zero partials.
template <bool FUSE>
__global__ void __launch_bounds__(BX * BY, 3)
batch_check_kernel(const BatchInst* __restrict__ insts, const BatchItem* __restrict__ items,
                   int n_items, double* __restrict__ partials) {
    __shared__ double tA[8], tB[8];
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const BatchItem it = items[w];
        const BatchInst* I = insts + it.inst;
        double acc[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
        const int active = I->active;
        const Lattice L = I->L;
        const Coef<double> C = I->C64;
        const int cur = I->cur;
        const double* s = I->s64[cur];
        double* s_new = I->s64[cur ^ 1];
        const float* d0 = I->delta[0];
        float* r32 = I->r32;
        __syncthreads();
        const int t = threadIdx.y * BX + threadIdx.x;
        if (t < 8) { tA[t] = I->C64.rA[t]; tB[t] = I->C64.rB[t]; }
        __syncthreads();
        if (active) {
            // the item's 1024 cells of the flattened plane, 4 a thread 256 cells apart
            // (consecutive threads on consecutive cells: coalesced)
            for (int q = 0; q < 4; ++q) {
                const int64_t cell = 4 * (int64_t)it.bx + 256 * q + t;
                if (cell < (int64_t)L.nxny)
                    check_column<FUSE, true>(L, C, tA, tB, s, d0, s_new, r32, acc,
                                             (int)(cell % L.nx), (int)(cell / L.nx), it.kb,
                                             it.ke);
            }
        }
        block_reduce_store(acc, partials + (int64_t)w * NRED);
    }
}

// Batched double-float check (FUSE: state = sdf[cur] + delta[0] written to sdf[cur ^ 1],
// FP32 forcing refreshed), one work item per loop trip: the work items of
// batch_check_kernel, the arithmetic of check_df_kernel. Items of inactive lattices write
// zero partials.
template <bool FUSE>
__global__ void __launch_bounds__(BX * BY, 3)
batch_check_df_kernel(const BatchInst* __restrict__ insts, const BatchItem* __restrict__ items,
                      int n_items, double* __restrict__ partials) {
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const BatchItem it = items[w];
        const BatchInst* I = insts + it.inst;
        float sum2 = 0.f, vmax = 0.f;
        int bad = 0;
        if (I->active) {   // uniform over the block
            const Lattice L = I->L;
            const L2F K = I->K2;
            const int cur = I->cur;
            const int t = threadIdx.y * BX + threadIdx.x;
            // the item's 1024 cells of the flattened plane, 4 a thread 256 cells apart
            for (int q = 0; q < 4; ++q) {
                const int64_t cell = 4 * (int64_t)it.bx + 256 * q + t;
                if (cell < (int64_t)L.nxny)
                    check_df_column<FUSE>(L, K, I->sdf[cur], I->delta[0], I->sdf[cur ^ 1],
                                          I->r32, 0, (int)(cell % L.nx), (int)(cell / L.nx),
                                          it.kb, it.ke, sum2, vmax, bad);
            }
        }
        double acc[NRED] = {(double)sum2, 0.0, 0.0, 0.0, 0.0, 0.0, (double)bad, (double)vmax};
        block_reduce_store(acc, partials + (int64_t)w * NRED);
    }
}

// Per-lattice sums of the item partials (one block per lattice, fixed order), then the
// convergence bookkeeping: residual = tau sqrt(sum r^2 / n_unknown); a lattice whose
// residual is <= tol (or that produced a non-finite value) becomes inactive. `fused`:
// the check just wrote s64[cur ^ 1], so active lattices flip cur first.
struct BatchCtl {
    double tol;
    double tau;
    double n_unknown;
    double residual;
    double sums[NRED];
    int64_t sweeps;
    int converged;
    int nonfinite;
};

__global__ void __launch_bounds__(256)
batch_finalize_kernel(BatchInst* __restrict__ insts, const int* __restrict__ item_begin,
                      const double* __restrict__ partials, BatchCtl* __restrict__ ctl,
                      int fused, int sweeps_done) {
    __shared__ double sh[256];
    const int q_inst = blockIdx.x;
    BatchInst& I = insts[q_inst];
    const int was_active = I.active;
    __syncthreads();
    if (!was_active) return;   // uniform per block
    const int b0 = item_begin[q_inst], b1 = item_begin[q_inst + 1];
    for (int q = 0; q < NRED; ++q) {
        const bool is_max = (q == NRED - 1);
        double a = 0.0;
        for (int b = b0 + threadIdx.x; b < b1; b += 256) {
            const double x = partials[(int64_t)b * NRED + q];
            a = is_max ? fmax(a, x) : a + x;
        }
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int sft = 128; sft > 0; sft >>= 1) {
            if (threadIdx.x < sft)
                sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + sft])
                                         : sh[threadIdx.x] + sh[threadIdx.x + sft];
            __syncthreads();
        }
        if (threadIdx.x == 0) ctl[q_inst].sums[q] = sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        BatchCtl& k = ctl[q_inst];
        if (fused) I.cur ^= 1;
        k.sweeps += sweeps_done;
        k.residual = k.n_unknown > 0 ? k.tau * sqrt(k.sums[0] / k.n_unknown) : 0.0;
        k.nonfinite = k.sums[6] > 0;
        if (k.residual <= k.tol || k.nonfinite) {
            k.converged = !k.nonfinite;
            I.active = 0;
        }
    }
}

// Largest diagonal of -L over unknown fluid cells (for dt = cfl / max d), and the
// per-cell local step dtc = cfl / d_c (rounded toward zero in FP32) when requested.
__global__ void __launch_bounds__(BX * BY)
diag_kernel(Lattice L, Coef<double> C, double cfl, float* __restrict__ dtc,
            double* __restrict__ partials, int kchunk) {
    RFB_LOAD_TABLES(double, C)
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    if (i < L.nx && j < L.ny) {
        const int kb = blockIdx.z * kchunk;
        const int ke = min(kb + kchunk, L.nz);
        const int nx = L.nx, nxny = L.nxny;
        int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
        for (int k = kb; k < ke; ++k, c += nxny) {
            const unsigned f = L.flags[c];
            if (!(f & F_FLUID) || (C.umt && (f & F_ELEC))) {
                if (dtc) dtc[c] = 0.0f;
                continue;
            }
            double uL = C.u[c];
            double uH = (i + 1 < nx) ? C.u[c + 1] : 0.0;
            double vL = C.v[c];
            double vH = (j + 1 < L.ny) ? C.v[c + nx] : 0.0;
            double wL = C.w[c], wH = C.w[c + nxny];
            const int nw = n_wall_of(f, i, j, k, nx, L.ny, L.nz);
            double mult = C.m ? C.m[c] : 1.0;
            double d = cell_diag<double>(C, tB, f, uL, uH, vL, vH, wL, wH, k == 0, nw, mult);
            acc[7] = fmax(acc[7], d);
            acc[0] = (acc[0] == 0.0 || d < acc[0]) ? d : acc[0];
            if (dtc) dtc[c] = d > 0.0 ? __double2float_rz(cfl / d) : 0.0f;
        }
    }
    // slot 0 carries a min: reduce it as -max(-x) by negating around the max slot
    __shared__ double mins[BX * BY];
    const int tid = threadIdx.y * BX + threadIdx.x;
    mins[tid] = acc[0] == 0.0 ? 1e300 : acc[0];
    acc[0] = 0.0;
    __syncthreads();
    for (int sft = BX * BY / 2; sft > 0; sft >>= 1) {
        if (tid < sft) mins[tid] = fmin(mins[tid], mins[tid + sft]);
        __syncthreads();
    }
    const double bmin = mins[0];
    __syncthreads();
    const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                        ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_reduce_store(acc, partials + bid * NRED);
    if (tid == 0) partials[bid * NRED + 0] = bmin;
}

__global__ void fill_kernel(double* __restrict__ a, double v, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        a[q] = v;
}

// Lattice statistics at creation, as per-block partials (fixed order with
// finalize_kernel): 0 fluid cells, 1 electrode cells, 2 sum of W over fluid inlet faces,
// 3 sum of W over fluid outlet faces, 4 count of area multipliers that are not finite
// and > 0 (m nullable). w: cell-aligned low-face W, N + nx*ny entries.
__global__ void __launch_bounds__(256)
stats_kernel(const uint8_t* __restrict__ flags, const double* __restrict__ w,
             const double* __restrict__ m, int64_t N, int64_t nxny,
             double* __restrict__ partials) {
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = flags[c];
        if (f & F_FLUID) {
            acc[0] += 1.0;
            if (f & F_ELEC) acc[1] += 1.0;
            if (c < nxny) acc[2] += w[c];
            if (c >= N - nxny) acc[3] += w[c + nxny];
        }
        if (m) {
            const double x = m[c];
            if (!(x > 0.0 && isfinite(x))) acc[4] += 1.0;
        }
    }
    block_reduce_store(acc, partials + (int64_t)blockIdx.x * NRED);
}

// Sum (slots 0..6) / max (slot 7) of the per-block partials, in a fixed order.
// min_slot0: slot 0 is reduced with min instead of a sum (diag_kernel).
__global__ void __launch_bounds__(256)
finalize_kernel(const double* __restrict__ partials, int64_t nblocks, double* __restrict__ out,
                int min_slot0) {
    __shared__ double sh[256];
    for (int q = 0; q < NRED; ++q) {
        const bool is_max = (q == NRED - 1);
        const bool is_min = (q == 0 && min_slot0);
        double a = is_min ? 1e300 : 0.0;
        for (int64_t b = threadIdx.x; b < nblocks; b += 256) {
            double x = partials[b * NRED + q];
            a = is_max ? fmax(a, x) : is_min ? fmin(a, x) : a + x;
        }
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int sft = 128; sft > 0; sft >>= 1) {
            if (threadIdx.x < sft) {
                double x = sh[threadIdx.x + sft];
                sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], x)
                                         : is_min ? fmin(sh[threadIdx.x], x)
                                                  : sh[threadIdx.x] + x;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sh[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// Setup kernels
// ---------------------------------------------------------------------------------

// flags (and the FP32 kernels' mask byte) from the solid mask (1 = fiber)
__global__ void flags_kernel(const uint8_t* __restrict__ solid, uint8_t* __restrict__ flags,
                             uint8_t* __restrict__ mask32, int nx, int ny, int nz) {
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((int64_t)nx * ny));
        const int64_t nxny = (int64_t)nx * ny;
        if (solid[c]) { flags[c] = 0; mask32[c] = 0; continue; }
        unsigned f = F_FLUID;
        int dom = 0, fl = 0;
        if (i > 0) { ++dom; if (!solid[c - 1]) { f |= F_XM; ++fl; } }
        if (i + 1 < nx) { ++dom; if (!solid[c + 1]) { f |= F_XP; ++fl; } }
        if (j > 0) { ++dom; if (!solid[c - nx]) { f |= F_YM; ++fl; } }
        if (j + 1 < ny) { ++dom; if (!solid[c + nx]) { f |= F_YP; ++fl; } }
        if (k > 0) { ++dom; if (!solid[c - nxny]) { f |= F_ZM; ++fl; } }
        if (k + 1 < nz) { ++dom; if (!solid[c + nxny]) { f |= F_ZP; ++fl; } }
        if (dom > fl) f |= F_ELEC;
        flags[c] = (uint8_t)f;
        mask32[c] = (uint8_t)(M_FLUID | (dom > fl ? M_ELEC : 0u) | ((unsigned)fl << 2) |
                              ((unsigned)(dom - fl) << 5));
    }
}

// Validate one face array against the mask and repack it cell aligned (low faces).
// axis 0: U (nx+1, ny, nz); 1: V (nx, ny+1, nz); 2: W (nx, ny, nz+1) -> N + nxny out.
// err[0]: non-finite; err[1]: nonzero on a wall/fiber face; err[2]: negative inlet or
// outlet velocity.
__global__ void repack_kernel(const double* __restrict__ in, const uint8_t* __restrict__ solid,
                              double* __restrict__ out, int nx, int ny, int nz, int axis,
                              unsigned long long* __restrict__ err) {
    const int ex = nx + (axis == 0), ey = ny + (axis == 1), ez = nz + (axis == 2);
    const int64_t M = (int64_t)ex * ey * ez;
    const int64_t nxny = (int64_t)nx * ny;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < M;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(q % ex);
        const int b = (int)((q / ex) % ey);
        const int k = (int)(q / ((int64_t)ex * ey));
        const double val = in[q];
        if (!isfinite(val)) atomicAdd(&err[0], 1ull);
        // the two cells sharing the face (either may be outside the domain)
        int i0 = a, j0 = b, k0 = k, i1 = a, j1 = b, k1 = k;
        int n_axis = axis == 0 ? nx : axis == 1 ? ny : nz;
        int pos = axis == 0 ? a : axis == 1 ? b : k;
        if (axis == 0) i0 = a - 1; else if (axis == 1) j0 = b - 1; else k0 = k - 1;
        bool lo_in = pos > 0, hi_in = pos < n_axis;
        bool lo_solid = lo_in && solid[i0 + nx * (int64_t)j0 + nxny * k0];
        bool hi_solid = hi_in && solid[i1 + nx * (int64_t)j1 + nxny * k1];
        bool wall = (axis != 2) && (!lo_in || !hi_in);
        if ((wall || lo_solid || hi_solid) && val != 0.0) atomicAdd(&err[1], 1ull);
        if (axis == 2 && (!lo_in || !hi_in) && val < 0.0) atomicAdd(&err[2], 1ull);
        if (axis == 0) {
            if (a < nx) out[a + nx * (int64_t)b + nxny * k] = val;
        } else if (axis == 1) {
            if (b < ny) out[a + nx * (int64_t)b + nxny * k] = val;
        } else {
            out[a + nx * (int64_t)b + nxny * k] = val;
        }
    }
}

// out64 = scale * in; out32 = (float) out64
__global__ void scale_kernel(const double* __restrict__ in, double* __restrict__ out64,
                             float* __restrict__ out32, double scale, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double x = scale * in[q];
        out64[q] = x;
        out32[q] = (float)x;
    }
}

// Initial state: s_in on unknown fluid cells, 1 on pinned electrode cells (U_mt), 0 on
// solid cells; written to both buffers.
__global__ void init_state_kernel(const uint8_t* __restrict__ flags, double* __restrict__ a,
                                  double* __restrict__ b, double s_in, int umt, int64_t n) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = flags[c];
        double x = 0.0;
        if (f & F_FLUID) x = (umt && (f & F_ELEC)) ? 1.0 : s_in;
        a[c] = x;
        if (b) b[c] = x;
    }
}

// s (both buffers) from a caller array; solid cells forced to 0 (pinned U_mt cells 1).
__global__ void set_state_kernel(const uint8_t* __restrict__ flags, const double* __restrict__ in,
                                 double* __restrict__ a, double* __restrict__ b,
                                 unsigned long long* __restrict__ err, int64_t n) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = flags[c];
        double x = (f & F_FLUID) ? in[c] : 0.0;
        if (!isfinite(x)) { atomicAdd(err, 1ull); x = 0.0; }
        a[c] = x;
        b[c] = x;
    }
}

// ---------------------------------------------------------------------------------
// Discrete adjoint of the steady state (FP64).
//
// The steady state solves L s + b = 0. For an objective J the adjoint solves
// L^T lam = -g with g = dJ/ds. Column c of L collects what cell c sends to its
// neighbours: through a face with outward velocity q > 0 the upwind flux q s_c leaves c
// and enters the neighbour, so
//   (L^T lam)_c = sum_{faces, q > 0} q (lam_nb - lam_c)      (outlet face: lam_nb = 0)
//               + D/h^2 sum_{fluid nbrs} (lam_nb - lam_c) - [inlet] gD/h^2 lam_c
//               - m_c kappa0(n_wall) B lam_c,
// i.e. the advection part gathers from downwind neighbours. The pseudo-time iteration
// lam <- lam + dt_c (L^T lam + g) uses the same dt_c as the forward one (L and L^T
// share their diagonal). Pinned U_mt cells are not unknowns: lam = 0 there.
// ---------------------------------------------------------------------------------
// The FP64 adjoint sweeps and checks are adjoint64c_kernel (the transpose gathered from
// the assembled operator); the mixed-precision ones sweep32v_kernel<*, true> and
// check_df_adjoint_kernel.

// g~ = dJ/ds / jscale on unknown fluid cells (0 elsewhere):
//   OBJ 0 (I_tot, U): m_c n_wall kR R~'(s_c)/K with kR = -k0 B / h (affine law, R~' = -B)
//                     or k0 K1 / h (mode 1, times g'(s_c));
//   OBJ 2 (U_mt):     [outlet] w_c / w_out_sum
__global__ void adjoint_source_kernel(Lattice L, Coef<double> C, int obj, double w_out_sum,
                                      double kR, const double* __restrict__ s,
                                      double* __restrict__ g) {
    const int64_t N = (int64_t)L.nxny * L.nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned f = L.flags[c];
        double x = 0.0;
        if ((f & F_FLUID) && !(C.umt && (f & F_ELEC))) {
            const int i = (int)(c % L.nx);
            const int j = (int)((c / L.nx) % L.ny);
            const int k = (int)(c / L.nxny);
            if (obj == 2) {
                if (k == L.nz - 1) x = C.w[c + L.nxny] / w_out_sum;
            } else {
                const int nw = n_wall_of(f, i, j, k, L.nx, L.ny, L.nz);
                x = (C.m ? C.m[c] : 1.0) * kR * nw;
                if (C.nl && nw > 0) x *= g_uniform_slope(s[c], C.alpha);
            }
        }
        g[c] = x;
    }
}

// Gradients at the steady state s with adjoint lam~ = lam / jscale:
//   dm[c] = jscale (mscale + lam~_c) kappa0(n_wall) R~(s_c)   (fluid cells, OBJ 0;
//           kappa0 R~ = n_wall (kap0A - kap0B s), or n_wall kap0A g(s) in mode 1)
//   slot 0 of the reduction: sum over unknown cells of lam~_c adv_c(s) (beta-scaled
//   velocities, so d/dbeta of RHS is adv/beta).
__global__ void __launch_bounds__(BX * BY)
gradient_kernel(Lattice L, Coef<double> C, const double* __restrict__ s,
                const double* __restrict__ lam, double kap0A, double kap0B, double jscale,
                double mscale, double* __restrict__ dm, double* __restrict__ partials,
                int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    __shared__ double tZ[8];
    if (threadIdx.y * BX + threadIdx.x < 8) tZ[threadIdx.y * BX + threadIdx.x] = 0.0;
    __syncthreads();
    if (i < L.nx && j < L.ny) {
        const int kb = blockIdx.z * kchunk;
        const int ke = min(kb + kchunk, L.nz);
        const int nx = L.nx, nxny = L.nxny;
        // advection only: no diffusion, no reaction
        Coef<double> A = C;
        A.Dh = 0.0;
        A.gDh = 0.0;
        int64_t c = (int64_t)i + (int64_t)nx * j + (int64_t)nxny * kb;
        double s_prev = kb > 0 ? s[c - nxny] : 0.0;
        double s_cur = s[c];
        double wL = C.w[c];
        for (int k = kb; k < ke; ++k, c += nxny) {
            const bool outlet = (k == L.nz - 1);
            double s_next = outlet ? 0.0 : s[c + nxny];
            double wH = C.w[c + nxny];
            const unsigned f = L.flags[c];
            double dmv = 0.0;
            if (f & F_FLUID) {
                const int nw = n_wall_of(f, i, j, k, nx, L.ny, L.nz);
                dmv = jscale * (mscale + lam[c]) * nw *
                      (C.nl ? kap0A * g_uniform(s_cur, C.alpha) : kap0A - kap0B * s_cur);
                if (!(C.umt && (f & F_ELEC))) {
                    double sxm = (f & F_XM) ? s[c - 1] : s_cur;
                    double sxp = (f & F_XP) ? s[c + 1] : s_cur;
                    double sym = (f & F_YM) ? s[c - nx] : s_cur;
                    double syp = (f & F_YP) ? s[c + nx] : s_cur;
                    double szm = (f & F_ZM) ? s_prev : s_cur;
                    double szp = (f & F_ZP) ? s_next : s_cur;
                    double uL = C.u[c];
                    double uH = (i + 1 < nx) ? C.u[c + 1] : 0.0;
                    double vL = C.v[c];
                    double vH = (j + 1 < L.ny) ? C.v[c + nx] : 0.0;
                    const double adv = cell_rhs<double>(A, tZ, tZ, s_cur, sxm, sxp, sym, syp,
                                                        szm, szp, uL, uH, vL, vH, wL, wH,
                                                        k == 0, outlet, 0, 0.0);
                    acc[0] += lam[c] * adv;
                }
            }
            if (dm) dm[c] = dmv;
            s_prev = s_cur;
            s_cur = s_next;
            wL = wH;
        }
    }
    const int64_t bid = (int64_t)blockIdx.x + (int64_t)gridDim.x *
                        ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_reduce_store(acc, partials + bid * NRED);
}

// 2x prolongation for iterative upsampling: a fine fluid cell takes its coarse parent's
// value (injection); if the parent is solid, the mean over the parent's fluid
// 6-neighbours (order -z, +z, -y, +y, -x, +x); if there are none, s_fill. Fine solid
// cells get 0. Written to both buffers of the fine state.
__global__ void prolong_kernel(const uint8_t* __restrict__ cflags, const double* __restrict__ sc,
                               int cnx, int cny, int cnz, const uint8_t* __restrict__ fflags,
                               double* __restrict__ fa, double* __restrict__ fb, double s_fill) {
    const int fnx = 2 * cnx, fny = 2 * cny;
    const int64_t fN = (int64_t)fnx * fny * (2 * cnz);
    const int64_t cnxny = (int64_t)cnx * cny;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < fN;
         q += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0;
        if (fflags[q] & F_FLUID) {
            const int i = (int)(q % fnx);
            const int j = (int)((q / fnx) % fny);
            const int k = (int)(q / ((int64_t)fnx * fny));
            const int ci = i >> 1, cj = j >> 1, ck = k >> 1;
            const int64_t p = ci + (int64_t)cnx * cj + cnxny * ck;
            if (cflags[p] & F_FLUID) {
                x = sc[p];
            } else {
                double acc = 0.0;
                int cnt = 0;
                if (ck > 0 && (cflags[p - cnxny] & F_FLUID)) { acc += sc[p - cnxny]; ++cnt; }
                if (ck + 1 < cnz && (cflags[p + cnxny] & F_FLUID)) { acc += sc[p + cnxny]; ++cnt; }
                if (cj > 0 && (cflags[p - cnx] & F_FLUID)) { acc += sc[p - cnx]; ++cnt; }
                if (cj + 1 < cny && (cflags[p + cnx] & F_FLUID)) { acc += sc[p + cnx]; ++cnt; }
                if (ci > 0 && (cflags[p - 1] & F_FLUID)) { acc += sc[p - 1]; ++cnt; }
                if (ci + 1 < cnx && (cflags[p + 1] & F_FLUID)) { acc += sc[p + 1]; ++cnt; }
                x = cnt ? acc / cnt : s_fill;
            }
        }
        fa[q] = x;
        fb[q] = x;
    }
}

}  // namespace rfb
