// FP32 correction sweeps with a stored per-cell step (local pseudo-time stepping).
//
// With the local step dt_c = C_CFL / d_c (d_c the diagonal of -L) one explicit update of
// the homogeneous correction equation is
//     delta'_c = (1 - C_CFL) delta_c
//              + dt_c (r_c + sum_f q_in,f delta_f + (D/h^2) sum_f delta_f),
// q_in,f the inflow through face f (beta/h times the face velocity where it points into
// the cell, else 0) and the sums over the six neighbours. The kernels evaluate it with
// the step distributed over the terms,
//     delta'_c = (1 - C_CFL) delta_c + dt_c r_c + sum_f a_f delta_f,
//     a_f = dt_c (q_in,f + D/h^2),
// so that the per-cell weights a_f and dt_c r_c, formed once per pass, make every further
// update of the cell seven FMAs. Solid and out-of-domain neighbours hold delta = 0 and
// their faces carry no velocity, so no face needs a mask test; cells that are not updated
// (solid, or electrode cells of U_mt) have dt_c = 0 and keep delta = 0, the value every
// correction cycle starts from. The step field is the one the FP64 path uses (written by
// the diagonal pass of every operating point), so the kernels stream the step instead of
// a mask byte and recompute no diagonal. For the transposed operator (adjoint
// corrections) the coefficient towards a neighbour is this cell's outflow through the
// shared face (the neighbour's inflow from it), with the same diagonal.
//
// sweep32d_kernel applies one sweep; sweep32tbd_kernel two sweeps per pass over HBM,
// planes staged by TMA through a three- or four-stage mbarrier ring (the scheme of
// sweep_tb.cuh, with the step plane in place of the mask plane; four stages keep three
// planes in flight and use 221 KB of shared memory). Both evaluate every update with
// dt_coef and dt_update below in the same operation order, so a pass is bitwise two
// sweeps.
#pragma once

#include "sweep_tb.cuh"

namespace rfb {

// Weights of one cell's update towards its neighbours -x, +x, -y, +y, -z, +z:
// a_f = dt (q_f + D/h^2), q_f the inflow through face f (TR: the outflow).
struct CoefD {
    float a[6];
};

template <bool TR>
__device__ __forceinline__ CoefD dt_coef(float dt, float Dh, float uL, float uH, float vL,
                                         float vH, float wL, float wH) {
    CoefD k;
    const float sg = TR ? -1.f : 1.f;
    const float dtD = dt * Dh;
    k.a[0] = fmaf(dt, fmaxf(sg * uL, 0.f), dtD);
    k.a[1] = fmaf(dt, fmaxf(-sg * uH, 0.f), dtD);
    k.a[2] = fmaf(dt, fmaxf(sg * vL, 0.f), dtD);
    k.a[3] = fmaf(dt, fmaxf(-sg * vH, 0.f), dtD);
    k.a[4] = fmaf(dt, fmaxf(sg * wL, 0.f), dtD);
    k.a[5] = fmaf(dt, fmaxf(-sg * wH, 0.f), dtD);
    return k;
}

// one update (omc = 1 - C_CFL, dtr = dt r)
__device__ __forceinline__ float dt_update(const CoefD& k, float omc, float sc, float dtr,
                                           float xm, float xp, float ym, float yp, float zm,
                                           float zp) {
    float acc = fmaf(omc, sc, dtr);
    acc = fmaf(k.a[0], xm, acc);
    acc = fmaf(k.a[1], xp, acc);
    acc = fmaf(k.a[2], ym, acc);
    acc = fmaf(k.a[3], yp, acc);
    acc = fmaf(k.a[4], zm, acc);
    acc = fmaf(k.a[5], zp, acc);
    return acc;
}

struct DArgs {
    int nx, ny, nz;
    int64_t nxny;
    const float* __restrict__ u;    // FP32 face velocities * beta / h (low faces)
    const float* __restrict__ v;
    const float* __restrict__ w;    // nz + 1 planes
    const float* __restrict__ dt;   // per-cell step (0: not updated)
    float omc, Dh;
};

// One sweep over the planes kb .. ke-1 of the columns (i0 .. i0+3, j), i0 % 4 == 0,
// nx % 4 == 0; every load of a plane is issued before its arithmetic.
template <bool TR>
__global__ void __launch_bounds__(VBX * VBY)
sweep32d_kernel(DArgs A, const float* __restrict__ s, float* __restrict__ s_out,
                const float* __restrict__ force, int kchunk) {
    const int i0 = 4 * (blockIdx.x * VBX + threadIdx.x);
    const int j = blockIdx.y * VBY + threadIdx.y;
    if (i0 >= A.nx || j >= A.ny) return;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, A.nz);
    const int nx = A.nx, nz = A.nz;
    const int64_t nxny = A.nxny;
    const bool has_xm = i0 > 0, has_xp = i0 + 4 < nx;
    const bool has_ym = j > 0, has_yp = j + 1 < A.ny;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t c = (int64_t)i0 + (int64_t)nx * j + nxny * kb;
    float4 d_prev = kb > 0 ? ldg4(s + c - nxny) : zero4;   // plane -1: outside, 0
    float4 d_cur = ldg4(s + c);
    float4 wL = ldg4(A.w + c);
    for (int k = kb; k < ke; ++k, c += nxny) {
        const float4 d_next = k == nz - 1 ? zero4 : ldg4(s + c + nxny);
        const float4 wH = ldg4(A.w + c + nxny);
        const float4 d_ym = has_ym ? ldg4(s + c - nx) : zero4;
        const float4 d_yp = has_yp ? ldg4(s + c + nx) : zero4;
        const float d_xm = has_xm ? __ldg(s + c - 1) : 0.f;
        const float d_xp = has_xp ? __ldg(s + c + 4) : 0.f;
        const float4 u4 = ldg4(A.u + c);
        const float u_nx = has_xp ? __ldg(A.u + c + 4) : 0.f;
        const float4 v4 = ldg4(A.v + c);
        const float4 vH4 = has_yp ? ldg4(A.v + c + nx) : zero4;
        const float4 r4 = ldg4(force + c);
        const float4 t4 = ldg4(A.dt + c);
        float out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const CoefD kc = dt_coef<TR>(el(t4, e), A.Dh, el(u4, e),
                                         e == 3 ? u_nx : el(u4, e + 1), el(v4, e), el(vH4, e),
                                         el(wL, e), el(wH, e));
            out[e] = dt_update(kc, A.omc, el(d_cur, e), el(t4, e) * el(r4, e),
                               e == 0 ? d_xm : el(d_cur, e - 1), e == 3 ? d_xp : el(d_cur, e + 1),
                               el(d_ym, e), el(d_yp, e), el(d_prev, e), el(d_next, e));
        }
        *reinterpret_cast<float4*>(s_out + c) = make_float4(out[0], out[1], out[2], out[3]);
        d_prev = d_cur;
        d_cur = d_next;
        wL = wH;
    }
}

// ---------------------------------------------------------------------------------
// Two sweeps per pass. Tile, staged boxes, thread layout, launch shapes and the bounded
// mbarrier waits are those of sweep32tb_kernel (sweep_tb.cuh); a stage holds six FP32
// planes (delta, forcing, u, v, w, step).
// ---------------------------------------------------------------------------------
// Tile geometry: TXI interior columns (128, or 64 for narrow lattices in batches), the 12
// interior rows of sweep_tb.cuh, boxes of TXI + 8 columns and 16 rows, one thread per 4
// cells of the box columns on 14 rows.
template <int TXI>
struct TBDGeom {
    static_assert(TXI % 4 == 0, "4-cell groups");
    static constexpr int BW = TXI + 8;           // staged columns
    static constexpr int GX = BW / 4;            // thread columns
    static constexpr int THREADS = GX * TB_GY;   // 476 (TXI = 128) or 252 (TXI = 64)
    static constexpr int PLANE = BW * TB_BH;
    static constexpr int F32 = PLANE * 4;        // bytes of one staged FP32 plane
    static constexpr int STAGE = 6 * F32;        // delta, forcing, u, v, w, step
    static_assert(F32 % 128 == 0, "stage buffers stay 128-B aligned");
};
static_assert(TBDGeom<128>::F32 == TB_F32 && TBDGeom<128>::THREADS == TB_THREADS, "geometry");
constexpr int TBD_STAGE = TBDGeom<128>::STAGE;
template <int NST, int TXI = 128>
__host__ __device__ constexpr int tbd_l1() { return NST * TBDGeom<TXI>::STAGE; }   // level-1 planes
template <int NST, int TXI = 128>
__host__ __device__ constexpr int tbd_bar() { return tbd_l1<NST, TXI>() + 2 * TBDGeom<TXI>::F32; }
template <int NST, int TXI = 128>
__host__ __device__ constexpr int tbd_smem() { return tbd_bar<NST, TXI>() + 64 + 128; }   // + slack
static_assert(tbd_smem<4>() <= 232448, "four stages fit the 227 KB a CTA may use");
static_assert(2 * tbd_smem<3, 64>() <= 233472, "two narrow three-stage CTAs fit an SM");

struct TBDArgs {
    int nx, ny, nz;
    int lc;                           // planes per z chunk (nz: one chunk)
    int64_t total;                    // tiles x chunks x lc (chunk-major, tile fastest)
    int64_t per;                      // planes of that space per CTA
    const float* __restrict__ d_in;   // delta read by this pass (prologue plane)
    float* __restrict__ d_out;
    float omc, Dh;
    unsigned int* err;                // set if a stage never arrives
};

// One lattice as the pass sees it: its six tensor maps (delta, forcing, u, v, w, step;
// generic addresses of kernel parameters or of global memory) and sizes.
struct TBDField {
    const CUtensorMap* d;
    const CUtensorMap* r;
    const CUtensorMap* u;
    const CUtensorMap* v;
    const CUtensorMap* w;
    const CUtensorMap* t;
    int nx, ny, nz;
    const float* d_in;                // delta read by this pass (prologue plane)
    float* d_out;
    float omc, Dh;
};

// Per-CTA state of the pass: the stage ring in shared memory, the parity of each stage's
// next completion and the stages with a copy in flight (every thread tracks the same).
template <int NST, int TXI = 128>
struct TBDRing {
    unsigned char* smem;
    uint64_t* bar;
    uint32_t phase, pend;
    unsigned int* err;
    __device__ __forceinline__ unsigned char* stage(int s) const {
        return smem + s * TBDGeom<TXI>::STAGE;
    }
    __device__ __forceinline__ bool wait(int s) {          // bounded wait for stage s
        if (!mbar_wait_bounded(&bar[s], (phase >> s) & 1u, TB_SPIN_LIMIT, err)) return false;
        phase ^= 1u << s;
        pend &= ~(1u << s);
        return true;
    }
};

template <int NST, int TXI = 128>
__device__ __forceinline__ TBDRing<NST, TXI> tbd_ring_init(unsigned char* smem_raw,
                                                           unsigned int* err) {
    TBDRing<NST, TXI> R;
    R.smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    R.bar = reinterpret_cast<uint64_t*>(R.smem + tbd_bar<NST, TXI>());
    R.phase = 0;
    R.pend = 0;
    R.err = err;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&R.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    return R;
}

// error path (a stage never arrived): wait, again with the limit, for the copies still
// in flight into this CTA's shared memory before the kernel returns
template <int NST, int TXI>
__device__ __forceinline__ void tbd_ring_drain(TBDRing<NST, TXI>& R) {
    for (int s = 0; s < NST; ++s)
        if (R.pend & (1u << s)) (void)R.wait(s);
}

// Two sweeps over planes kb .. ke-1 of one tile of lattice F, from F.d_in into F.d_out.
// Every stage issued is waited for, so the ring is empty when it returns; false if a
// wait gave up (the CTA decides together at its step barrier).
template <bool TR, int NST, int TXI = 128>
__device__ __forceinline__ bool tbd_segment(TBDRing<NST, TXI>& R, const TBDField& F, int tile,
                                            int kb, int ke) {
    using G = TBDGeom<TXI>;
    const int tid = threadIdx.x;
    const int tx = tid % G::GX, ty = tid / G::GX;
    const int bxx = 4 * tx, byy = 1 + ty;              // this thread's cells in the box
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const bool interior = tx >= 1 && tx < 1 + TXI / 4 && ty >= 1 && ty <= TB_TYI;
    const int64_t nxny = (int64_t)nx * ny;
    const int o = byy * G::BW + bxx;                   // offset in a staged plane
    const int gx = (nx + TXI - 1) / TXI;
    const float omc = F.omc, Dh = F.Dh;
    unsigned char* smem = R.smem;
    const int x0 = TXI * (tile % gx) - 4;           // box origin (4-cell aligned)
    const int y0 = TB_TYI * (tile / gx) - 2;
    const int i0 = x0 + bxx, j = y0 + byy;
    const bool in_dom = i0 >= 0 && i0 < nx && j >= 0 && j < ny;
    auto issue = [&](int p, int s) {                   // plane p -> stage s
        R.pend |= 1u << s;
        if (tid != 0) return;                          // one thread issues the copies
        unsigned char* S = R.stage(s);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&R.bar[s], G::STAGE);
        tma_load_3d(S, F.d, x0, y0, p, &R.bar[s]);
        tma_load_3d(S + G::F32, F.r, x0, y0, p, &R.bar[s]);
        tma_load_3d(S + 2 * G::F32, F.u, x0, y0, p, &R.bar[s]);
        tma_load_3d(S + 3 * G::F32, F.v, x0, y0, p, &R.bar[s]);
        tma_load_3d(S + 4 * G::F32, F.w, x0, y0, p, &R.bar[s]);
        tma_load_3d(S + 5 * G::F32, F.t, x0, y0, p, &R.bar[s]);
    };
    __syncthreads();   // the previous segment's readers are done with every stage
    for (int s = 0; s < NST; ++s) issue(kb - 1 + s, s);                 // kb-1, kb, ...

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 l1_m2 = zero4, l1_m1 = zero4;               // own level 1 at z-2, z-1
    // Two register sets that swap roles every step (the loop is unrolled by two):
    // weights, step times forcing and own level-0 value of the step's plane (written) and
    // of the plane before it (read).
    CoefD kcA[4], kcB[4];
    float4 rA = zero4, rB = zero4, dA = zero4, dB = zero4;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        for (int s = 0; s < 6; ++s) kcB[e].a[s] = 0.f;
    if (in_dom && kb >= 2) dB = ldg4(F.d_in + i0 + (int64_t)nx * j + nxny * (kb - 2));
    bool good = R.wait(0);
    int s0 = 0;                                        // stage holding plane z

    auto step = [&](int z, CoefD (&kc)[4], float4& rr, float4& dc,
                    const CoefD (&pkc)[4], const float4& prr, const float4& pdc) -> bool {
        const int s1 = s0 == NST - 1 ? 0 : s0 + 1;
        if (good) good = R.wait(s1);
        const float* D0 = reinterpret_cast<const float*>(R.stage(s0));
        const float* R0 = D0 + G::PLANE;
        const float* U0 = R0 + G::PLANE;
        const float* V0 = U0 + G::PLANE;
        const float* W0 = V0 + G::PLANE;
        const float* T0 = W0 + G::PLANE;
        const float* D1 = reinterpret_cast<const float*>(R.stage(s1));
        const float* W1 = D1 + 4 * G::PLANE;
        // ---- level 1 at plane z
        dc = lds4(D0 + o);
        const float4 dn = lds4(D1 + o);
        const float4 u4 = lds4(U0 + o);
        const float un = U0[o + 4];
        const float4 v4 = lds4(V0 + o);
        const float4 vh4 = lds4(V0 + o + G::BW);
        const float4 wl4 = lds4(W0 + o);
        const float4 wh4 = lds4(W1 + o);
        const float4 t4 = lds4(T0 + o);
        const float4 r4 = lds4(R0 + o);
        rr = make_float4(t4.x * r4.x, t4.y * r4.y, t4.z * r4.z, t4.w * r4.w);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            kc[e] = dt_coef<TR>(el(t4, e), Dh, el(u4, e), e == 3 ? un : el(u4, e + 1),
                                el(v4, e), el(vh4, e), el(wl4, e), el(wh4, e));
        float4 l1 = dc;
        if (in_dom && z >= 0 && z < nz) {
            const float dxm = D0[o - 1], dxp = D0[o + 4];
            const float4 dym = lds4(D0 + o - G::BW), dyp = lds4(D0 + o + G::BW);
            float out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                out[e] = dt_update(kc[e], omc, el(dc, e), el(rr, e),
                                   e == 0 ? dxm : el(dc, e - 1), e == 3 ? dxp : el(dc, e + 1),
                                   el(dym, e), el(dyp, e), el(pdc, e), el(dn, e));
            l1 = make_float4(out[0], out[1], out[2], out[3]);
        }
        float* L1w = reinterpret_cast<float*>(smem + tbd_l1<NST, TXI>()) + (z & 1) * G::PLANE;
        *reinterpret_cast<float4*>(L1w + o) = l1;
        // ---- level 2 at plane z-1 (its level-1 neighbours were stored last step)
        const int zz = z - 1;
        if (zz >= kb && interior && in_dom) {
            const float* L1r =
                reinterpret_cast<const float*>(smem + tbd_l1<NST, TXI>()) + (zz & 1) * G::PLANE;
            const float lxm = L1r[o - 1], lxp = L1r[o + 4];
            const float4 lym = lds4(L1r + o - G::BW), lyp = lds4(L1r + o + G::BW);
            float out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                out[e] = dt_update(pkc[e], omc, el(l1_m1, e), el(prr, e),
                                   e == 0 ? lxm : el(l1_m1, e - 1),
                                   e == 3 ? lxp : el(l1_m1, e + 1), el(lym, e), el(lyp, e),
                                   el(l1_m2, e), el(l1, e));
            *reinterpret_cast<float4*>(F.d_out + i0 + (int64_t)nx * j + nxny * zz) =
                make_float4(out[0], out[1], out[2], out[3]);
        }
        l1_m2 = l1_m1;
        l1_m1 = l1;
        // ---- all threads are done with stage s0: refill it with plane z + NST
        if (!__syncthreads_and(good)) return false;
        if (z + NST <= ke + 1) issue(z + NST, s0);
        s0 = s1;
        return true;
    };

    for (int z = kb - 1; z <= ke; z += 2) {
        if (!step(z, kcA, rA, dA, kcB, rB, dB)) return false;
        if (z + 1 > ke) break;
        if (!step(z + 1, kcB, rB, dB, kcA, rA, dA)) return false;
    }
    return true;
}

// One pass over one lattice: this CTA's share of the linear index
// ((chunk * tiles + tile) * lc + plane in chunk), walked as one z segment per
// (chunk, tile) item it touches; positions past nz in the last chunk are skipped. With
// one chunk and per = tiles * nz / CTAs this is a persistent launch with equal shares;
// with per = lc every CTA takes one item and neighbouring tiles run together.
template <bool TR, int NST>
__global__ void __launch_bounds__(TB_THREADS, 1)
sweep32tbd_kernel(const __grid_constant__ CUtensorMap tm_d, const __grid_constant__ CUtensorMap tm_r,
                  const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
                  const __grid_constant__ CUtensorMap tm_w, const __grid_constant__ CUtensorMap tm_t,
                  TBDArgs A) {
    extern __shared__ unsigned char smem_raw[];
    TBDRing<NST> R = tbd_ring_init<NST>(smem_raw, A.err);
    const TBDField F{&tm_d, &tm_r, &tm_u, &tm_v, &tm_w, &tm_t, A.nx, A.ny, A.nz,
                     A.d_in, A.d_out, A.omc, A.Dh};
    const int gx = (A.nx + TB_TXI - 1) / TB_TXI;
    const int tiles = gx * ((A.ny + TB_TYI - 1) / TB_TYI);
    const int64_t q1 = min((int64_t)(blockIdx.x + 1) * A.per, A.total);
    bool ok = true;
    for (int64_t q = (int64_t)blockIdx.x * A.per; q < q1 && ok;) {
        const int64_t item = q / A.lc;
        const int zl = (int)(q % A.lc);
        const int tile = (int)(item % tiles);
        const int kb = (int)(item / tiles) * A.lc + zl;
        const int64_t item_end = (item + 1) * A.lc;
        if (kb >= A.nz) { q = item_end; continue; }   // padding of a short last chunk
        const int ke = (int)min((int64_t)A.nz, kb + (min(q1, item_end) - q));
        q = min(q1, item_end);
        ok = tbd_segment<TR, NST>(R, F, tile, kb, ke);
    }
    if (!ok) tbd_ring_drain<NST>(R);
}

// ---------------------------------------------------------------------------------
// Batched two-sweep pass: many lattices in one launch. Work items are (lattice, tile, z
// chunk), lattice-major with neighbouring tiles of a chunk next to each other; one CTA per
// SM walks the item list in a fixed round-robin order. Each lattice's tensor maps live
// in global memory (written by the host before the launch); lattices that have converged
// are skipped (their flag is read from the batch's descriptors, which the check kernels
// update), so a captured graph keeps working as lattices drop out.
// ---------------------------------------------------------------------------------
struct BatchTBD {
    CUtensorMap td[2];                // delta buffer 0 and 1
    CUtensorMap tr, tu, tv, tw, tt;   // forcing, u, v, w, step
    int nx, ny, nz, pad_;
    float omc, Dh;
};

struct BatchTBItem {
    int inst, tile, kb, ke;           // planes kb .. ke-1 of one tile of one lattice
};

template <int NST, int TXI>
__global__ void __launch_bounds__(TBDGeom<TXI>::THREADS, TXI == 64 ? 2 : 1)
batch_tbd_kernel(const BatchTBD* __restrict__ lat, const BatchInst* __restrict__ insts,
                 const BatchTBItem* __restrict__ items, int n_items, int parity,
                 unsigned int* err) {
    extern __shared__ unsigned char smem_raw[];
    TBDRing<NST, TXI> R = tbd_ring_init<NST, TXI>(smem_raw, err);
    bool ok = true;
    for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        const BatchTBItem it = items[w];
        const BatchInst* I = insts + it.inst;
        if (!I->active) continue;   // uniform over the CTA
        const BatchTBD* L = lat + it.inst;
        const TBDField F{&L->td[parity], &L->tr, &L->tu, &L->tv, &L->tw, &L->tt, L->nx, L->ny,
                         L->nz, I->delta[parity], I->delta[parity ^ 1], L->omc, L->Dh};
        ok = tbd_segment<false, NST, TXI>(R, F, it.tile, it.kb, it.ke);
    }
    if (!ok) tbd_ring_drain<NST>(R);
}

}  // namespace rfb
