// Three FP32 correction sweeps per pass over HBM (local steps), with the per-cell update
// coefficients of the two older levels kept in tensor memory.
//
// The pass extends the two-sweep scheme of sweep_dt.cuh by one level. A CTA owns an x-y
// tile of 128 x 10 cells, stages 136 x 16 boxes (4 halo columns, 3 halo rows on each
// side) and marches z; at step z it computes
//   - level 1 (one sweep) at plane z for the 136 x 14 box rows 1..14, from the staged
//     level-0 planes z, z+1 and its own level-0 value at z-1 (registers), and stores it in
//     a double-buffered shared plane;
//   - level 2 at plane z-1 for box rows 2..13 from the level-1 plane z-1 (shared), its own
//     level-1 values at z-2, z (registers), into a second double-buffered shared plane;
//   - level 3 at plane z-2 for the 128 x 10 interior from the level-2 plane z-2 (shared)
//     and its own level-2 values at z-3, z-1, written to HBM.
// A level-l value is valid l cells inside the box, so the 4 halo columns and 3 halo rows
// leave the interior exact after three sweeps.
//
// Each level needs the update weights of its plane (a_f and dt r, sweep_dt.cuh). Level 1
// derives them from the staged planes; the staged plane is then released, and the 28
// words of a thread's four cells are stored in tensor memory (tcgen05.st, 32 lanes x 32
// columns per warp), from where levels 2 and 3 load them one and two steps later
// (tcgen05.ld). Tensor memory (256 KB per SM, unused by this pass otherwise) thus holds
// three planes of weights that would not fit next to the staged planes in shared memory
// nor in the register file at 480 threads. The 4 threads past the 476 that own cells
// repeat the first four cell groups of the last row, so that every thread runs the same
// instructions; they store nothing.
//
// Staging: delta and w (read at planes z and z+1) go through one mbarrier ring of NA
// stages, forcing, u, v and step (read at plane z only) through a second ring of NB = 3
// stages, so both keep two planes in flight while the CTA works on plane z.
//
// Every update is dt_coef and dt_update with the same operands in the same order as the
// one-sweep kernel, so a pass is bitwise three sweeps.
#pragma once

#include "sweep_dt.cuh"

namespace rfb {

constexpr int T3_TYI = 10;                    // interior rows of a tile
constexpr int T3_THREADS = 480;               // 476 cell threads (34 x 14) + 4: whole warps
static_assert(T3_THREADS >= TB_THREADS && T3_THREADS % 32 == 0, "whole warps");
constexpr int T3_ASTAGE = 2 * TB_F32;         // delta, w
constexpr int T3_BSTAGE = 4 * TB_F32;         // forcing, u, v, step
constexpr int T3_NB = 3;
template <int NA> __host__ __device__ constexpr int t3_l1() { return NA * T3_ASTAGE + T3_NB * T3_BSTAGE; }
template <int NA> __host__ __device__ constexpr int t3_l2() { return t3_l1<NA>() + 2 * TB_F32; }
template <int NA> __host__ __device__ constexpr int t3_bar() { return t3_l2<NA>() + 2 * TB_F32; }
template <int NA> __host__ __device__ constexpr int t3_tslot() { return t3_bar<NA>() + 64; }
template <int NA> __host__ __device__ constexpr int t3_smem() { return t3_tslot<NA>() + 16 + 128; }
static_assert(t3_smem<5>() <= 232448, "five delta stages fit the 227 KB a CTA may use");
static_assert(4 + T3_NB <= 8, "barriers fit their 64 bytes");
// tensor memory: warps w and w + 4 share a lane quarter; each warp holds three slots of 32
// columns, so the 15 warps use 4 x 96 columns of the 512 allocated (a power of two)
constexpr uint32_t T3_TMEM_COLS = 512;
constexpr int T3_SLOT_COLS = 32;
static_assert(((T3_THREADS / 32 + 3) / 4) * 3 * T3_SLOT_COLS <= (int)T3_TMEM_COLS,
              "the coefficient slots fit the allocation");

// ---- tensor memory (tcgen05) helpers
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 32 consecutive columns of this thread's lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// load, then wait for the load; the wait names the registers so that no use of them is
// scheduled before it
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                   "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                   "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]),
                   "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                   "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]),
                   "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

// the words of four cells: seven per cell (six weights a_f, then dt r), four unused
__device__ __forceinline__ void t3_pack(const CoefD (&kc)[4], const float (&dtr)[4],
                                        uint32_t (&v)[32]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int f = 0; f < 6; ++f) v[7 * e + f] = __float_as_uint(kc[e].a[f]);
        v[7 * e + 6] = __float_as_uint(dtr[e]);
    }
    v[28] = v[29] = v[30] = v[31] = 0u;
}
__device__ __forceinline__ CoefD t3_coef(const uint32_t (&v)[32], int e) {
    CoefD k;
#pragma unroll
    for (int f = 0; f < 6; ++f) k.a[f] = __uint_as_float(v[7 * e + f]);
    return k;
}
__device__ __forceinline__ float t3_dtr(const uint32_t (&v)[32], int e) {
    return __uint_as_float(v[7 * e + 6]);
}

// Stage rings: NA (delta, w) stages, then T3_NB (forcing, u, v, step) stages; barrier q
// of stage q of the first ring, NA + q of the second.
template <int NA>
struct T3Ring {
    unsigned char* smem;
    uint64_t* bar;
    uint32_t phase, pend;
    unsigned int* err;
    __device__ __forceinline__ unsigned char* a(int s) const { return smem + s * T3_ASTAGE; }
    __device__ __forceinline__ unsigned char* b(int s) const {
        return smem + NA * T3_ASTAGE + s * T3_BSTAGE;
    }
    __device__ __forceinline__ bool wait(int q) {
        if (!mbar_wait_bounded(&bar[q], (phase >> q) & 1u, TB_SPIN_LIMIT, err)) return false;
        phase ^= 1u << q;
        pend &= ~(1u << q);
        return true;
    }
    __device__ __forceinline__ void drain() {
        for (int q = 0; q < NA + T3_NB; ++q)
            if (pend & (1u << q)) (void)wait(q);
    }
};

// Three sweeps over planes kb .. ke-1 of one tile of lattice F, from F.d_in into F.d_out;
// tmem is this warp's first coefficient column in its lane quarter. Every stage issued is
// waited for; false if a wait gave up (decided by the CTA together at its step barrier).
template <bool TR, int NA>
__device__ __forceinline__ bool t3_segment(T3Ring<NA>& R, const TBDField& F, uint32_t tmem,
                                           int tile, int kb, int ke) {
    const int tid0 = threadIdx.x;
    const bool act = tid0 < TB_THREADS;                // the last 4 threads store nothing
    const int tid = act ? tid0 : tid0 - TB_GX;         // ... and repeat row 13's first groups
    const int tx = tid % TB_GX, ty = tid / TB_GX;
    const int bxx = 4 * tx, byy = 1 + ty;              // this thread's cells in the box
    const bool lv2 = act && ty >= 1 && ty <= 12;       // box rows 2 .. 13
    const bool lv3 = act && tx >= 1 && tx <= TB_TXI / 4 && ty >= 2 && ty <= 11;
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const int64_t nxny = (int64_t)nx * ny;
    const int o = byy * TB_BW + bxx;                   // offset in a staged plane
    const int gx = (nx + TB_TXI - 1) / TB_TXI;
    const float omc = F.omc, Dh = F.Dh;
    const int x0 = TB_TXI * (tile % gx) - 4;           // box origin (4-cell aligned)
    const int y0 = T3_TYI * (tile / gx) - 3;
    const int i0 = x0 + bxx, j = y0 + byy;
    const bool in_dom = i0 >= 0 && i0 < nx && j >= 0 && j < ny;
    float* L1 = reinterpret_cast<float*>(R.smem + t3_l1<NA>());
    float* L2 = reinterpret_cast<float*>(R.smem + t3_l2<NA>());
    auto issue_a = [&](int p, int s) {                 // delta, w of plane p -> stage s
        R.pend |= 1u << s;
        if (tid0 != 0) return;
        unsigned char* S = R.a(s);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&R.bar[s], T3_ASTAGE);
        tma_load_3d(S, F.d, x0, y0, p, &R.bar[s]);
        tma_load_3d(S + TB_F32, F.w, x0, y0, p, &R.bar[s]);
    };
    auto issue_b = [&](int p, int s) {                 // forcing, u, v, step -> stage s
        R.pend |= 1u << (NA + s);
        if (tid0 != 0) return;
        unsigned char* S = R.b(s);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&R.bar[NA + s], T3_BSTAGE);
        tma_load_3d(S, F.r, x0, y0, p, &R.bar[NA + s]);
        tma_load_3d(S + TB_F32, F.u, x0, y0, p, &R.bar[NA + s]);
        tma_load_3d(S + 2 * TB_F32, F.v, x0, y0, p, &R.bar[NA + s]);
        tma_load_3d(S + 3 * TB_F32, F.t, x0, y0, p, &R.bar[NA + s]);
    };
    // planes read: delta and w kb-2 .. ke+2, the others kb-2 .. ke+1
    const int zf = kb - 2;
    __syncthreads();   // the previous segment's readers are done with every stage
    for (int s = 0; s < NA; ++s)
        if (zf + s <= ke + 2) issue_a(zf + s, s);
    for (int s = 0; s < T3_NB; ++s)
        if (zf + s <= ke + 1) issue_b(zf + s, s);

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pdc = zero4;                                // own level 0 at z-1
    float4 l1_m2 = zero4, l1_m1 = zero4;               // own level 1 at z-2, z-1
    float4 l2_m2 = zero4, l2_m1 = zero4;               // own level 2 at z-3, z-2
    if (in_dom && zf >= 1) pdc = ldg4(F.d_in + i0 + (int64_t)nx * j + nxny * (zf - 1));
    bool good = R.wait(0);
    int a0 = 0, b0 = 0;                                // stages holding plane z
    int sl0 = 0, sl1 = 2, sl2 = 1;                     // weight slots of z, z-1, z-2

    for (int z = zf; z <= ke + 1; ++z) {
        const int a1 = a0 == NA - 1 ? 0 : a0 + 1;
        if (good) good = R.wait(a1);                   // delta, w of plane z+1
        if (good) good = R.wait(NA + b0);              // forcing, u, v, step of plane z
        // ---- level 1 at plane z
        const float* D0 = reinterpret_cast<const float*>(R.a(a0));
        const float* W0 = D0 + TB_PLANE;
        const float* D1 = reinterpret_cast<const float*>(R.a(a1));
        const float* W1 = D1 + TB_PLANE;
        const float* R0 = reinterpret_cast<const float*>(R.b(b0));
        const float* U0 = R0 + TB_PLANE;
        const float* V0 = U0 + TB_PLANE;
        const float* T0 = V0 + TB_PLANE;
        const float4 dc = lds4(D0 + o);
        float4 l1 = dc;
        {
            const float4 dn = lds4(D1 + o);
            const float4 u4 = lds4(U0 + o);
            const float un = U0[o + 4];
            const float4 v4 = lds4(V0 + o);
            const float4 vh4 = lds4(V0 + o + TB_BW);
            const float4 wl4 = lds4(W0 + o);
            const float4 wh4 = lds4(W1 + o);
            const float4 t4 = lds4(T0 + o);
            const float4 r4 = lds4(R0 + o);
            CoefD kc[4];
            float dtr[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                kc[e] = dt_coef<TR>(el(t4, e), Dh, el(u4, e), e == 3 ? un : el(u4, e + 1),
                                    el(v4, e), el(vh4, e), el(wl4, e), el(wh4, e));
                dtr[e] = el(t4, e) * el(r4, e);
            }
            if (in_dom && z >= 0 && z < nz) {
                const float dxm = D0[o - 1], dxp = D0[o + 4];
                const float4 dym = lds4(D0 + o - TB_BW), dyp = lds4(D0 + o + TB_BW);
                float out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    out[e] = dt_update(kc[e], omc, el(dc, e), dtr[e],
                                       e == 0 ? dxm : el(dc, e - 1),
                                       e == 3 ? dxp : el(dc, e + 1), el(dym, e), el(dyp, e),
                                       el(pdc, e), el(dn, e));
                l1 = make_float4(out[0], out[1], out[2], out[3]);
            }
            if (act) *reinterpret_cast<float4*>(L1 + (z & 1) * TB_PLANE + o) = l1;
            uint32_t kw[32];
            t3_pack(kc, dtr, kw);
            tmem_st32(tmem + sl0 * T3_SLOT_COLS, kw);
        }
        // ---- level 2 at plane z-1 (the level-1 plane z-1 was stored last step)
        float4 l2 = l1_m1;                             // rows without level 2 keep level 1
        if (z >= kb) {
            uint32_t kw[32];
            tmem_ld32(tmem + sl1 * T3_SLOT_COLS, kw);
            const int zz = z - 1;
            if (lv2) {
                if (in_dom && zz >= 0 && zz < nz) {
                    const float* P = L1 + (zz & 1) * TB_PLANE;
                    const float lxm = P[o - 1], lxp = P[o + 4];
                    const float4 lym = lds4(P + o - TB_BW), lyp = lds4(P + o + TB_BW);
                    float out[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        out[e] = dt_update(t3_coef(kw, e), omc, el(l1_m1, e), t3_dtr(kw, e),
                                           e == 0 ? lxm : el(l1_m1, e - 1),
                                           e == 3 ? lxp : el(l1_m1, e + 1), el(lym, e),
                                           el(lyp, e), el(l1_m2, e), el(l1, e));
                    l2 = make_float4(out[0], out[1], out[2], out[3]);
                }
                *reinterpret_cast<float4*>(L2 + (zz & 1) * TB_PLANE + o) = l2;
            }
        }
        // ---- level 3 at plane z-2 (the level-2 plane z-2 was stored last step)
        if (z >= kb + 2) {
            uint32_t kw[32];
            tmem_ld32(tmem + sl2 * T3_SLOT_COLS, kw);
            const int zz = z - 2;                      // kb <= zz < ke <= nz
            if (lv3 && in_dom) {
                const float* P = L2 + (zz & 1) * TB_PLANE;
                const float lxm = P[o - 1], lxp = P[o + 4];
                const float4 lym = lds4(P + o - TB_BW), lyp = lds4(P + o + TB_BW);
                float out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    out[e] = dt_update(t3_coef(kw, e), omc, el(l2_m1, e), t3_dtr(kw, e),
                                       e == 0 ? lxm : el(l2_m1, e - 1),
                                       e == 3 ? lxp : el(l2_m1, e + 1), el(lym, e), el(lyp, e),
                                       el(l2_m2, e), el(l2, e));
                *reinterpret_cast<float4*>(F.d_out + i0 + (int64_t)nx * j + nxny * zz) =
                    make_float4(out[0], out[1], out[2], out[3]);
            }
        }
        pdc = dc;
        l1_m2 = l1_m1;
        l1_m1 = l1;
        l2_m2 = l2_m1;
        l2_m1 = l2;
        // ---- this step's weights are in tensor memory, and all threads are done with
        // the stages of plane z: refill them
        tmem_wait_st();
        if (!__syncthreads_and(good)) return false;
        if (z + NA <= ke + 2) issue_a(z + NA, a0);
        if (z + T3_NB <= ke + 1) issue_b(z + T3_NB, b0);
        a0 = a1;
        b0 = b0 == T3_NB - 1 ? 0 : b0 + 1;
        const int s_free = sl2;                        // plane z-2's slot: plane z+1's
        sl2 = sl1;
        sl1 = sl0;
        sl0 = s_free;
    }
    return true;
}

// One three-sweep pass over one lattice; the work split is that of sweep32tbd_kernel
// (persistent equal shares or one (tile, z chunk) item per CTA) over 128 x 10 tiles.
template <bool TR, int NA>
__global__ void __launch_bounds__(T3_THREADS, 1)
sweep32t3_kernel(const __grid_constant__ CUtensorMap tm_d, const __grid_constant__ CUtensorMap tm_r,
                 const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
                 const __grid_constant__ CUtensorMap tm_w, const __grid_constant__ CUtensorMap tm_t,
                 TBDArgs A) {
    extern __shared__ unsigned char smem_raw[];
    T3Ring<NA> R;
    R.smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    R.bar = reinterpret_cast<uint64_t*>(R.smem + t3_bar<NA>());
    R.phase = 0;
    R.pend = 0;
    R.err = A.err;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(R.smem + t3_tslot<NA>());
    const int warp = threadIdx.x / 32;
    if (warp == 0) {
        tmem_alloc(tslot, T3_TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < NA + T3_NB; ++q) mbar_init(&R.bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *tslot;
    // lane quarter warp % 4 (bits 31:16 of the address), columns by warp / 4
    const uint32_t tmem = tbase + ((uint32_t)(32 * (warp & 3)) << 16) +
                          (uint32_t)((warp >> 2) * 3 * T3_SLOT_COLS);
    const TBDField F{&tm_d, &tm_r, &tm_u, &tm_v, &tm_w, &tm_t, A.nx, A.ny, A.nz,
                     A.d_in, A.d_out, A.omc, A.Dh};
    const int gx = (A.nx + TB_TXI - 1) / TB_TXI;
    const int tiles = gx * ((A.ny + T3_TYI - 1) / T3_TYI);
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
        ok = t3_segment<TR, NA>(R, F, tmem, tile, kb, ke);
    }
    if (!ok) R.drain();
    // every warp's tensor-memory accesses are complete before the columns are released
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, T3_TMEM_COLS);
}

}  // namespace rfb
