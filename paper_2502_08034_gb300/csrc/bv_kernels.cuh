// Device code of the Butler-Volmer model with electromigration (Sec. II.C; the steady
// form of Algorithm 2), FP64.
//
// Unknowns on fluid cells: the oxidised and reduced quinone O, R (charge -2, diffusivity
// D), protons H (+1, D_H) and the electrolyte potential phi; the counter-ion HSO4- (X,
// -1, D_X) follows from electroneutrality, C_X = C_H - 2 (C_O + C_R). Per species j:
//   RHS_j = advection (first-order upwind, inlet value C_j,in on the inlet face,
//           zero-gradient outlet) + diffusion (D_j / h^2 to fluid neighbours, 2 D_j / h^2
//           towards the inlet face) + migration + n_j S,
//   migration = g_j [sum_n (C_c + C_n)/2 (phi_n - phi_c) + 2 C_c (0 - phi_c) through the
//           membrane (low-x face of i = 0; protons only)],  g_j = z_j D_j F / (R T h^2),
//   S = k0 a_c (C_O e^{alpha V_c} - C_R e^{(alpha-1) V_c}),  V_c = V~ + n_e phi_c / V_T
// (Eqs. source-term-bv1 and etat-from-s-bv; n_O = -1, n_R = +1, n_H = -2). Potential
// (Eq. poisson-phi in Algorithm 2's form div(kappa grad phi)):
//   sum_n kappa_f (phi_n - phi_c)/h^2 - 2 kappa_m,c phi_c / h^2 = n_e F S
//        - F sum_k z_k D_k lap_h C_k,
//   kappa_f = (F^2/RT) sum_k z_k^2 D_k (C_k,c + C_k,n)/2, kappa_m,c = (F^2/RT) D_H C_H,c,
// so the sum of z_k F times the species fluxes over a cell's faces is the potential
// equation: the discrete charge balance.
//
// Species: explicit pseudo-time sweeps at a fixed potential, each species with its own
// local step C_CFL / d_j,c (d_j,c: outflow + diffusion diagonal + |migration diagonal| +
// the source's slope in C_j); potential: Jacobi-preconditioned conjugate gradients on the
// SPD operator -K with device-resident scalars (no host round trip per iteration).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "soc_kernels.cuh"

namespace rfb {

constexpr int BV_TPB = 256;
constexpr int BV_NB = 152 * 8;   // blocks of the grid-stride reductions

struct BVSpecies {
    double Dh;     // D_j / h^2
    double gDh;    // inlet face: 2 D_j / h^2 (face reading) or D_j / h^2 (ghost)
    double g;      // z_j D_j F / (R T h^2)
    double c_in;   // inlet concentration
    double nst;    // stoichiometric number
    double zD;     // z_j D_j (potential equation)
    int membrane;  // crosses the membrane (protons)
};

struct BVArgs {
    int nx, ny, nz;
    int64_t nxny, N;
    const uint8_t* __restrict__ flags;
    const double* __restrict__ u;   // beta/h * face velocity (low faces; w: nz+1 planes)
    const double* __restrict__ v;
    const double* __restrict__ w;
    const double* __restrict__ m;   // area multiplier or nullptr
    BVSpecies sp[3];                // O, R, H
    double x_zD, x_cin; // counter-ion: z D, inlet concentration
    double lap_in;      // inlet face weight of lap_h: 2 (value on the face) or 1 (ghost)
    double kap0;        // k0 / h
    double alpha, Vt, ne_VT;   // transfer coefficient, V~, n_e / V_T
    double F, pre;      // Faraday's constant, F^2 / (R T)
    double D4;          // sum over the quinones of z^2 D: 4 D (both species)
    double D_H, D_X;    // for kappa
    double ne_F;        // n_e F
    double h2;          // h^2
    double cfl;
};

struct BVCell {         // neighbour layout of one fluid cell
    int64_t n[6];       // neighbour indices (-x, +x, -y, +y, -z, +z), -1 if not fluid
    double q[6];        // outward face velocity * beta / h (+x, +y, +z positive outward)
    bool inlet, outlet, membrane;
    int nw, nf;         // fiber neighbours, fluid neighbours
};

__device__ __forceinline__ BVCell bv_cell(const BVArgs& A, int64_t c, unsigned f) {
    BVCell b;
    const int i = (int)(c % A.nx);
    const int j = (int)((c / A.nx) % A.ny);
    const int k = (int)(c / A.nxny);
    b.n[0] = (f & F_XM) ? c - 1 : -1;
    b.n[1] = (f & F_XP) ? c + 1 : -1;
    b.n[2] = (f & F_YM) ? c - A.nx : -1;
    b.n[3] = (f & F_YP) ? c + A.nx : -1;
    b.n[4] = (f & F_ZM) ? c - A.nxny : -1;
    b.n[5] = (f & F_ZP) ? c + A.nxny : -1;
    b.q[0] = -A.u[c];
    b.q[1] = (i + 1 < A.nx) ? A.u[c + 1] : 0.0;
    b.q[2] = -A.v[c];
    b.q[3] = (j + 1 < A.ny) ? A.v[c + A.nx] : 0.0;
    b.q[4] = -A.w[c];
    b.q[5] = A.w[c + A.nxny];
    b.inlet = (k == 0);
    b.outlet = (k == A.nz - 1);
    b.membrane = (i == 0);
    b.nw = n_wall_of(f, i, j, k, A.nx, A.ny, A.nz);
    b.nf = __popc(f & F_NBRS);
    return b;
}

// Net rate of change of species j at cell c and the diagonal of its step.
__device__ __forceinline__ double bv_species_rhs(const BVArgs& A, const BVSpecies& P,
                                                 const BVCell& b, const double* __restrict__ C,
                                                 const double* __restrict__ phi, int64_t c,
                                                 double src, double* diag) {
    const double cc = C[c];
    const double pc = phi[c];
    double adv = 0.0, out = 0.0, dif = 0.0, mig = 0.0, mdiag = 0.0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const double q = b.q[f];
        const int64_t n = b.n[f];
        double cn;
        if (n >= 0) cn = C[n];
        else if (f == 4 && b.inlet) cn = P.c_in;    // inflow through the inlet face
        else cn = cc;                                // outlet (zero gradient) or closed
        // outward flux q * (upwind value)
        if (q > 0.0) { adv -= q * cc; out += q; }
        else adv -= q * cn;
        if (n >= 0) {
            dif += cn - cc;
            const double dp = phi[n] - pc;
            mig += 0.5 * (cc + cn) * dp;
            mdiag += 0.5 * dp;
        }
    }
    double rhs = adv + P.Dh * dif;
    double d = out + P.Dh * (double)b.nf;
    if (b.inlet) { rhs += P.gDh * (P.c_in - cc); d += P.gDh; }
    if (P.membrane && b.membrane) { mig += 2.0 * cc * (0.0 - pc); mdiag -= 2.0 * pc; }
    rhs += P.g * mig + P.nst * src;
    d += fabs(P.g * mdiag);
    *diag = d;
    return rhs;
}

// source and its slopes in C_O (kf) and C_R (kb) at cell c
__device__ __forceinline__ double bv_source(const BVArgs& A, const BVCell& b, int64_t c,
                                            double cO, double cR, double pc, double* kf,
                                            double* kb) {
    const double kap = A.kap0 * (A.m ? A.m[c] : 1.0) * (double)b.nw;
    const double vc = A.Vt + A.ne_VT * pc;
    *kf = kap * exp(A.alpha * vc);
    *kb = kap * exp((A.alpha - 1.0) * vc);
    return *kf * cO - *kb * cR;
}

// One explicit step of the three species at the potential phi (ping-pong buffers).
__global__ void __launch_bounds__(BV_TPB)
bv_sweep_kernel(BVArgs A, const double* __restrict__ O, const double* __restrict__ R,
                const double* __restrict__ H, const double* __restrict__ phi,
                double* __restrict__ O2, double* __restrict__ R2, double* __restrict__ H2) {
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < A.N;
         c += (int64_t)gridDim.x * BV_TPB) {
        const unsigned f = A.flags[c];
        if (!(f & F_FLUID)) continue;
        const BVCell b = bv_cell(A, c, f);
        double kf, kb;
        const double S = bv_source(A, b, c, O[c], R[c], phi[c], &kf, &kb);
        double d;
        double r = bv_species_rhs(A, A.sp[0], b, O, phi, c, S, &d);
        O2[c] = O[c] + A.cfl / (d + kf) * r;
        r = bv_species_rhs(A, A.sp[1], b, R, phi, c, S, &d);
        R2[c] = R[c] + A.cfl / (d + kb) * r;
        r = bv_species_rhs(A, A.sp[2], b, H, phi, c, S, &d);
        H2[c] = H[c] + A.cfl / d * r;
    }
}

// Residual pass at (C, phi): per block sums of RHS_O^2, RHS_R^2, RHS_H^2, S (slots 0-3),
// the outlet's sum of W C_R / (C_O + C_R) and of W (4, 5), the protons' migration current
// density sum through the membrane (6), and the largest |right-hand side of the potential
// equation| (7, a max). Also writes the potential equation's right-hand side
// (n_e F S - F sum_k z_k D_k lap C_k), the cell conductivity kappa_c and the membrane
// conductivity for the conjugate gradients.
__global__ void __launch_bounds__(BV_TPB)
bv_check_kernel(BVArgs A, const double* __restrict__ O, const double* __restrict__ R,
                const double* __restrict__ H, const double* __restrict__ phi,
                double* __restrict__ bphi, double* __restrict__ kcell,
                double* __restrict__ kmem, double* __restrict__ partials) {
    double acc[NRED];
#pragma unroll
    for (int q = 0; q < NRED; ++q) acc[q] = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < A.N;
         c += (int64_t)gridDim.x * BV_TPB) {
        const unsigned f = A.flags[c];
        if (!(f & F_FLUID)) {
            bphi[c] = 0.0;
            kcell[c] = 0.0;
            kmem[c] = 0.0;
            continue;
        }
        const BVCell b = bv_cell(A, c, f);
        const double cO = O[c], cR = R[c], cH = H[c], pc = phi[c];
        double kf, kb, d;
        const double S = bv_source(A, b, c, cO, cR, pc, &kf, &kb);
        const double rO = bv_species_rhs(A, A.sp[0], b, O, phi, c, S, &d);
        const double rR = bv_species_rhs(A, A.sp[1], b, R, phi, c, S, &d);
        const double rH = bv_species_rhs(A, A.sp[2], b, H, phi, c, S, &d);
        acc[0] += rO * rO;
        acc[1] += rR * rR;
        acc[2] += rH * rH;
        acc[3] += S;
        if (b.outlet) {
            const double wq = b.q[5];
            acc[4] += wq * cR / (cO + cR);
            acc[5] += wq;
        }
        // lap_h of each species (fluid neighbours, inlet face term)
        double lap[3] = {0.0, 0.0, 0.0}, lapX = 0.0;
        const double cX = cH - 2.0 * (cO + cR);
#pragma unroll
        for (int f6 = 0; f6 < 6; ++f6) {
            const int64_t n = b.n[f6];
            if (n < 0) continue;
            const double nO = O[n], nR = R[n], nH = H[n];
            lap[0] += nO - cO;
            lap[1] += nR - cR;
            lap[2] += nH - cH;
            lapX += (nH - 2.0 * (nO + nR)) - cX;
        }
        double ion = 0.0;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            double l = lap[s];
            if (b.inlet) l += A.lap_in * (A.sp[s].c_in - (s == 0 ? cO : s == 1 ? cR : cH));
            ion += A.sp[s].zD * l;
        }
        if (b.inlet) lapX += A.lap_in * (A.x_cin - cX);
        ion += A.x_zD * lapX;
        const double bp = A.ne_F * S - A.F * ion / A.h2;
        bphi[c] = bp;
        acc[NRED - 1] = fmax(acc[NRED - 1], fabs(bp));
        kcell[c] = A.pre * (A.D4 * (cO + cR) + A.D_H * cH + A.D_X * cX);
        kmem[c] = b.membrane ? A.pre * A.D_H * cH : 0.0;
        if (b.membrane) acc[6] += A.pre * A.D_H * cH * 2.0 * (0.0 - pc);
    }
    block_reduce_store(acc, partials + (int64_t)blockIdx.x * NRED);
}

// (A x)_c with A = -K: sum_n kappa_f (x_c - x_n)/h^2 + 2 kappa_m,c x_c / h^2
__device__ __forceinline__ double bv_apply(const BVArgs& A, const double* __restrict__ kcell,
                                           const double* __restrict__ kmem,
                                           const double* __restrict__ x, int64_t c,
                                           unsigned f, double* diag) {
    const double kc = kcell[c], xc = x[c];
    double a = 0.0, dg = 0.0;
    const int64_t nb[6] = {(f & F_XM) ? c - 1 : -1, (f & F_XP) ? c + 1 : -1,
                           (f & F_YM) ? c - A.nx : -1, (f & F_YP) ? c + A.nx : -1,
                           (f & F_ZM) ? c - A.nxny : -1, (f & F_ZP) ? c + A.nxny : -1};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (nb[q] < 0) continue;
        const double kf = 0.5 * (kc + kcell[nb[q]]);
        a += kf * (xc - x[nb[q]]);
        dg += kf;
    }
    a += 2.0 * kmem[c] * xc;
    dg += 2.0 * kmem[c];
    *diag = dg / A.h2;
    return a / A.h2;
}

// CG scalars in device memory: 0 rz, 1 pq, 2 rz_new
// start: r = -bphi - A x, z = r / diag, p = z; partial sums of r.z (slot 0)
__global__ void __launch_bounds__(BV_TPB)
bv_cg_start_kernel(BVArgs A, const double* __restrict__ kcell, const double* __restrict__ kmem,
                   const double* __restrict__ bphi, const double* __restrict__ x,
                   double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
                   double* __restrict__ dinv, double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < A.N;
         c += (int64_t)gridDim.x * BV_TPB) {
        const unsigned f = A.flags[c];
        double rv = 0.0, di = 0.0;
        if (f & F_FLUID) {
            double dg;
            const double ax = bv_apply(A, kcell, kmem, x, c, f, &dg);
            rv = -bphi[c] - ax;
            di = dg > 0.0 ? 1.0 / dg : 0.0;
        }
        r[c] = rv;
        dinv[c] = di;
        z[c] = rv * di;
        p[c] = rv * di;
        acc += rv * rv * di;
    }
    __shared__ double sh[BV_TPB / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < BV_TPB / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__device__ __forceinline__ void bv_block_sum_store(double acc, double* out) {
    __shared__ double sh[BV_TPB / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < BV_TPB / 32; ++w) s += sh[w];
        *out = s;
    }
}

// fixed-order sum of n block partials into *out (one block)
__global__ void bv_sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double sh[BV_TPB];
    double a = 0.0;
    for (int b = threadIdx.x; b < n; b += BV_TPB) a += part[b];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = BV_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// q = A p, partial sums of p.q
__global__ void __launch_bounds__(BV_TPB)
bv_cg_matvec_kernel(BVArgs A, const double* __restrict__ kcell, const double* __restrict__ kmem,
                    const double* __restrict__ p, double* __restrict__ q,
                    double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < A.N;
         c += (int64_t)gridDim.x * BV_TPB) {
        const unsigned f = A.flags[c];
        double a = 0.0;
        if (f & F_FLUID) {
            double dg;
            a = bv_apply(A, kcell, kmem, p, c, f, &dg);
        }
        q[c] = a;
        acc += p[c] * a;
    }
    bv_block_sum_store(acc, part + blockIdx.x);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = dinv r; partial sums of r.z
__global__ void __launch_bounds__(BV_TPB)
bv_cg_update_kernel(int64_t N, const double* __restrict__ sc, double* __restrict__ x,
                    double* __restrict__ r, double* __restrict__ z, const double* __restrict__ p,
                    const double* __restrict__ q, const double* __restrict__ dinv,
                    double* __restrict__ part) {
    const double pq = sc[1];
    const double alpha = pq != 0.0 ? sc[0] / pq : 0.0;
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * BV_TPB) {
        x[c] += alpha * p[c];
        const double rv = r[c] - alpha * q[c];
        r[c] = rv;
        const double zv = dinv[c] * rv;
        z[c] = zv;
        acc += rv * zv;
    }
    bv_block_sum_store(acc, part + blockIdx.x);
}

// beta = rz_new / rz; p = z + beta p; then rz <- rz_new (one thread, after the grid)
__global__ void __launch_bounds__(BV_TPB)
bv_cg_direction_kernel(int64_t N, const double* __restrict__ sc, double* __restrict__ p,
                       const double* __restrict__ z) {
    const double beta = sc[0] != 0.0 ? sc[2] / sc[0] : 0.0;
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * BV_TPB)
        p[c] = z[c] + beta * p[c];
}

__global__ void bv_copy_scalar_kernel(double* __restrict__ sc) { sc[0] = sc[2]; }

// Per block (BV_STATS values): max over fluid cells of |(-bphi - A x)_c| (0), of
// |x_c - x_old_c| (1), sum (2), min (3) and max (4) of x, and max of diag_c |x_c| (5), the
// size of the terms whose rounding bounds how small the residual can get.
constexpr int BV_STATS = 6;
__global__ void __launch_bounds__(BV_TPB)
bv_potential_stats_kernel(BVArgs A, const double* __restrict__ kcell,
                          const double* __restrict__ kmem, const double* __restrict__ bphi,
                          const double* __restrict__ x, const double* __restrict__ x_old,
                          double* __restrict__ part) {
    double res = 0.0, dx = 0.0, sum = 0.0, mn = INFINITY, mx = -INFINITY, tm = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < A.N;
         c += (int64_t)gridDim.x * BV_TPB) {
        const unsigned f = A.flags[c];
        if (!(f & F_FLUID)) continue;
        double dg;
        const double ax = bv_apply(A, kcell, kmem, x, c, f, &dg);
        res = fmax(res, fabs(-bphi[c] - ax));
        dx = fmax(dx, fabs(x[c] - x_old[c]));
        tm = fmax(tm, dg * fabs(x[c]));
        sum += x[c];
        mn = fmin(mn, x[c]);
        mx = fmax(mx, x[c]);
    }
    __shared__ double sh[BV_STATS][BV_TPB / 32];
    for (int o = 16; o > 0; o >>= 1) {
        tm = fmax(tm, __shfl_down_sync(0xffffffffu, tm, o));
        res = fmax(res, __shfl_down_sync(0xffffffffu, res, o));
        dx = fmax(dx, __shfl_down_sync(0xffffffffu, dx, o));
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = res; sh[1][w] = dx; sh[2][w] = sum; sh[3][w] = mn; sh[4][w] = mx;
        sh[5][w] = tm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double o[BV_STATS] = {sh[0][0], sh[1][0], sh[2][0], sh[3][0], sh[4][0], sh[5][0]};
        for (int q = 1; q < BV_TPB / 32; ++q) {
            o[0] = fmax(o[0], sh[0][q]); o[1] = fmax(o[1], sh[1][q]); o[2] += sh[2][q];
            o[3] = fmin(o[3], sh[3][q]); o[4] = fmax(o[4], sh[4][q]); o[5] = fmax(o[5], sh[5][q]);
        }
        for (int q = 0; q < BV_STATS; ++q) part[(int64_t)blockIdx.x * BV_STATS + q] = o[q];
    }
}

// initial state from an SBV state s (model refinement) or from s_in (s == nullptr)
__global__ void bv_init_kernel(BVArgs A, const double* __restrict__ s, double s_in, double c0,
                               double* __restrict__ O, double* __restrict__ R,
                               double* __restrict__ H, double* __restrict__ phi) {
    for (int64_t c = blockIdx.x * (int64_t)BV_TPB + threadIdx.x; c < A.N;
         c += (int64_t)gridDim.x * BV_TPB) {
        const bool fl = A.flags[c] & F_FLUID;
        const double sc = s ? s[c] : s_in;
        O[c] = fl ? (1.0 - sc) * c0 : 0.0;
        R[c] = fl ? sc * c0 : 0.0;
        H[c] = fl ? A.sp[2].c_in - 2.0 * (sc * c0 - A.sp[1].c_in) : 0.0;
        phi[c] = 0.0;
    }
}

}  // namespace rfb
