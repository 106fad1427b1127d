// Temporally blocked FP32 correction sweep for sm_103a: two pseudo-time steps per pass
// over HBM, z-planes staged into shared memory by TMA (cp.async.bulk.tensor) through a
// three-stage mbarrier ring.
//
// A CTA owns an x-y tile of 128 x 12 cells and marches z. The FP32 fields are staged as
// 136 x 16 boxes (4 halo columns and 2 halo rows on each side; a 32-bit TMA box starts on
// a multiple of 4 cells), the 8-bit mask as a 160 x 16 box (16 halo columns: an 8-bit box
// starts on a multiple of 16 cells). At step z the CTA
//   - computes level 1 (one sweep) at plane z from the staged level-0 planes z, z+1 and
//     its own level-0 value at z-1 kept in registers, for every cell of the tile and a
//     one-cell ring around it, and stores it in a double-buffered shared plane;
//   - computes level 2 (the second sweep) at plane z-1 for the 128 x 12 interior from the
//     level-1 plane z-1 (shared), its own level-1 values at z-2, z, and the coefficients of
//     plane z-1 kept in registers from the previous step; level 2 is written to HBM.
// Per pass each cell's delta, forcing, three face velocities and mask byte are read once
// and delta is written once, for two sweeps. The per-cell arithmetic is cell_update32,
// the same function as the one-sweep kernel: a pass is bitwise two plain sweeps.
#pragma once

#include <cuda.h>

#include "soc_kernels.cuh"

namespace rfb {

constexpr int TB_TXI = 128;                    // interior columns of a tile
constexpr int TB_TYI = 12;                     // interior rows of a tile
constexpr int TB_BW = TB_TXI + 8;              // staged FP32 columns: 4 halo + 128 + 4 halo
constexpr int TB_BWM = TB_TXI + 32;            // staged mask columns: 16 + 128 + 16
constexpr int TB_BH = TB_TYI + 4;              // staged rows: 2 halo + 12 + 2 halo
constexpr int TB_GX = TB_BW / 4;               // 34 groups of 4 cells: columns [-4, 132)
constexpr int TB_GY = TB_TYI + 2;              // 14 rows of threads: rows [-1, 13)
// 476 threads (15 warps): 128 registers a thread fit in the register file
constexpr int TB_THREADS = TB_GX * TB_GY;
constexpr int TB_PLANE = TB_BW * TB_BH;        // 2176 cells per staged FP32 plane
constexpr int TB_F32 = TB_PLANE * 4;           // 8704 bytes (68 x 128)
constexpr int TB_MPLANE = TB_BWM * TB_BH;      // 2560 mask bytes (20 x 128)
constexpr int TB_STAGE = 5 * TB_F32 + TB_MPLANE;
constexpr int TB_NSTAGE = 3;
constexpr int TB_L1 = TB_NSTAGE * TB_STAGE;    // offset of the two level-1 planes
constexpr int TB_BAR = TB_L1 + 2 * TB_F32;     // offset of the stage barriers
constexpr int TB_SMEM = TB_BAR + 64 + 128;     // + alignment slack for the base
constexpr uint32_t TB_TX_BYTES = 5 * TB_F32 + TB_MPLANE;
static_assert(TB_F32 % 128 == 0 && TB_MPLANE % 128 == 0, "stage buffers stay 128-B aligned");
constexpr unsigned long long TB_SPIN_LIMIT = 1ull << 26;   // bounded mbarrier waits

struct TBArgs {
    int nx, ny, nz;
    int lc;                           // planes per z chunk (nz: one chunk)
    int64_t total;                    // tiles x chunks x lc (chunk-major, tile fastest)
    int64_t per;                      // planes of that space per CTA
    const float* __restrict__ d_in;   // delta read by this pass (prologue plane)
    float* __restrict__ d_out;
    float Dh, gDh, dt, cfl;
    int umt;
    float tB[8];
    unsigned int* err;                // set if a stage never arrives
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of `bar` with the given parity, polling at most `limit` times; on
// giving up, set *err and return false (a wait never blocks a kernel indefinitely).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit, unsigned int* err) {
    for (unsigned long long n = 0; !mbar_try_wait(bar, parity);) {
        if (++n > limit) {
            atomicExch(err, 1u);
            return false;
        }
    }
    return true;
}

// Self-test of the bounded wait: one CTA waits on a barrier that no thread or copy ever
// completes; every thread must give up after `limit` polls and set *err; *done is set
// after the block's barrier, showing that the kernel ran to its end.
__global__ void mbar_timeout_probe_kernel(unsigned long long limit, unsigned int* err,
                                          unsigned int* done) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool arrived = mbar_wait_bounded(&bar, 0u, limit, err);
    __syncthreads();
    if (threadIdx.x == 0 && !arrived) atomicExch(done, 1u);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

template <bool LOCAL_DT>
__global__ void __maxnreg__(128)
sweep32tb_kernel(const __grid_constant__ CUtensorMap tm_d, const __grid_constant__ CUtensorMap tm_r,
                 const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v,
                 const __grid_constant__ CUtensorMap tm_w, const __grid_constant__ CUtensorMap tm_f,
                 TBArgs A) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + TB_BAR);
    __shared__ float tB[8];
    __shared__ float tdf[DFIX_TABLE];
    const int tid = threadIdx.x;
    if (tid < 8) tB[tid] = A.tB[tid];
    __syncthreads();
    build_dfix_table(tdf, tB, A.umt, A.Dh, A.gDh, tid, TB_THREADS);   // read after the
                                                                     // barrier below
    const int tx = tid % TB_GX, ty = tid / TB_GX;
    const int bxx = 4 * tx, byy = 1 + ty;              // this thread's cells in the box
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const bool interior = tx >= 1 && tx < 1 + TB_TXI / 4 && ty >= 1 && ty <= TB_TYI;
    const int64_t nxny = (int64_t)nx * ny;
    const int o = byy * TB_BW + bxx;                   // offset in a staged FP32 plane
    const int om = byy * TB_BWM + 12 + bxx;            // offset in the staged mask plane
    const int gx = (nx + TB_TXI - 1) / TB_TXI;

    auto stage = [&](int s) { return smem + s * TB_STAGE; };
    uint32_t phase = 0;   // parity of each stage's next completion
    uint32_t pend = 0;    // stages with a load in flight (every thread tracks the same set)
    auto wait = [&](int s) -> bool {                   // bounded wait for stage s
        if (!mbar_wait_bounded(&bar[s], (phase >> s) & 1u, TB_SPIN_LIMIT, A.err)) return false;
        phase ^= 1u << s;
        pend &= ~(1u << s);
        return true;
    };

    if (tid == 0) {
        for (int s = 0; s < TB_NSTAGE; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // This CTA's share of the work: positions q0 .. q1-1 of the linear index
    // ((chunk * tiles + tile) * lc + plane in chunk), walked as one z segment per
    // (chunk, tile) item it touches; positions past nz in the last chunk are skipped.
    // With one chunk and per = tiles * nz / CTAs this is a persistent launch with equal
    // shares; with per = lc every CTA takes one item and neighbouring tiles run together.
    // Every segment waits for each stage it issues, so the ring is empty between segments.
    const int tiles = gx * ((ny + TB_TYI - 1) / TB_TYI);
    const int64_t q1 = min((int64_t)(blockIdx.x + 1) * A.per, A.total);
    bool ok = true;
    for (int64_t q = (int64_t)blockIdx.x * A.per; q < q1 && ok;) {
        const int64_t item = q / A.lc;
        const int zl = (int)(q % A.lc);
        const int tile = (int)(item % tiles);
        const int kb = (int)(item / tiles) * A.lc + zl;
        const int64_t item_end = (item + 1) * A.lc;
        if (kb >= nz) { q = item_end; continue; }     // padding of a short last chunk
        const int ke = (int)min((int64_t)nz, kb + (min(q1, item_end) - q));
        q = min(q1, item_end);   // the rest of an item past nz is padding
        const int x0 = TB_TXI * (tile % gx) - 4;       // FP32 box origin (4-cell aligned)
        const int y0 = TB_TYI * (tile / gx) - 2;
        const int i0 = x0 + bxx, j = y0 + byy;
        const bool in_dom = i0 >= 0 && i0 < nx && j >= 0 && j < ny;
        auto issue = [&](int p, int s) {               // plane p -> stage s
            pend |= 1u << s;
            if (tid != 0) return;                      // one thread issues the copies
            unsigned char* S = stage(s);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[s], TB_TX_BYTES);
            tma_load_3d(S, &tm_d, x0, y0, p, &bar[s]);
            tma_load_3d(S + TB_F32, &tm_r, x0, y0, p, &bar[s]);
            tma_load_3d(S + 2 * TB_F32, &tm_u, x0, y0, p, &bar[s]);
            tma_load_3d(S + 3 * TB_F32, &tm_v, x0, y0, p, &bar[s]);
            tma_load_3d(S + 4 * TB_F32, &tm_w, x0, y0, p, &bar[s]);
            tma_load_3d(S + 5 * TB_F32, &tm_f, x0 - 12, y0, p, &bar[s]);   // 16-aligned
        };
        __syncthreads();   // the previous segment's readers are done with every stage
        for (int s = 0; s < TB_NSTAGE; ++s) issue(kb - 1 + s, s);       // kb-1, kb, kb+1

        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 l1_m2 = zero4, l1_m1 = zero4;           // own level 1 at z-2, z-1
        // Two register sets that swap roles every step (the loop below is unrolled by two,
        // so nothing is copied): update coefficients, forcing and own level-0 value of the
        // step's plane (written) and of the plane before it (read).
        Coef32 kcA[4], kcB[4];
        float4 rA = zero4, rB = zero4, dA = zero4, dB = zero4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            for (int s = 0; s < 6; ++s) kcB[e].a[s] = 0.f;
            kcB[e].ac = 1.f;
            kcB[e].dt = 0.f;
        }
        if (in_dom && kb >= 2) dB = ldg4(A.d_in + i0 + (int64_t)nx * j + nxny * (kb - 2));
        // A wait that gives up leaves this thread's `good` false; the CTA decides together
        // at the step's barrier (so no thread is left at a barrier the others skipped).
        bool good = wait(0);
        int s0 = 0;                                    // stage holding plane z

        auto step = [&](int z, Coef32 (&kc)[4], float4& rr, float4& dc,
                        const Coef32 (&pkc)[4], const float4& prr, const float4& pdc) -> bool {
            const int s1 = s0 == TB_NSTAGE - 1 ? 0 : s0 + 1;
            if (good) good = wait(s1);
            const float* D0 = reinterpret_cast<const float*>(stage(s0));
            const float* R0 = D0 + TB_PLANE;
            const float* U0 = R0 + TB_PLANE;
            const float* V0 = U0 + TB_PLANE;
            const float* W0 = V0 + TB_PLANE;
            const unsigned char* F0 = reinterpret_cast<const unsigned char*>(W0 + TB_PLANE);
            const float* D1 = reinterpret_cast<const float*>(stage(s1));
            const float* W1 = D1 + 4 * TB_PLANE;
            // ---- level 1 at plane z
            dc = lds4(D0 + o);
            const float4 dn = lds4(D1 + o);
            const float4 u4 = lds4(U0 + o);
            const float un = U0[o + 4];
            const float4 v4 = lds4(V0 + o);
            const float4 vh4 = lds4(V0 + o + TB_BW);
            const float4 wl4 = lds4(W0 + o);
            const float4 wh4 = lds4(W1 + o);
            rr = lds4(R0 + o);
            const uint32_t f4 = *reinterpret_cast<const uint32_t*>(F0 + om);
            // the cells' update coefficients for plane z, used by level 1 now and by
            // level 2 at the next step
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const unsigned m = (f4 >> (8 * e)) & 0xffu;
                kc[e] = cell_coef32<LOCAL_DT>(tdf[(z == 0 ? 256 : 0) + m], el(u4, e),
                                              e == 3 ? un : el(u4, e + 1), el(v4, e),
                                              el(vh4, e), el(wl4, e), el(wh4, e), A.Dh, A.cfl,
                                              A.dt);
            }
            float4 l1 = dc;
            if (in_dom && z >= 0 && z < nz) {
                const float dxm = D0[o - 1], dxp = D0[o + 4];
                const float4 dym = lds4(D0 + o - TB_BW), dyp = lds4(D0 + o + TB_BW);
                float out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    out[e] = cell_apply32(kc[e], el(dc, e), e == 0 ? dxm : el(dc, e - 1),
                                          e == 3 ? dxp : el(dc, e + 1), el(dym, e), el(dyp, e),
                                          el(pdc, e), el(dn, e), el(rr, e));
                l1 = make_float4(out[0], out[1], out[2], out[3]);
            }
            float* L1w = reinterpret_cast<float*>(smem + TB_L1) + (z & 1) * TB_PLANE;
            *reinterpret_cast<float4*>(L1w + o) = l1;
            // ---- level 2 at plane z-1 (its level-1 neighbours were stored last step)
            const int zz = z - 1;
            if (zz >= kb && interior && in_dom) {
                const float* L1r =
                    reinterpret_cast<const float*>(smem + TB_L1) + (zz & 1) * TB_PLANE;
                const float lxm = L1r[o - 1], lxp = L1r[o + 4];
                const float4 lym = lds4(L1r + o - TB_BW), lyp = lds4(L1r + o + TB_BW);
                float out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    out[e] = cell_apply32(pkc[e], el(l1_m1, e), e == 0 ? lxm : el(l1_m1, e - 1),
                                          e == 3 ? lxp : el(l1_m1, e + 1), el(lym, e),
                                          el(lyp, e), el(l1_m2, e), el(l1, e), el(prr, e));
                *reinterpret_cast<float4*>(A.d_out + i0 + (int64_t)nx * j + nxny * zz) =
                    make_float4(out[0], out[1], out[2], out[3]);
            }
            l1_m2 = l1_m1;
            l1_m1 = l1;
            // ---- all threads are done with stage s0: refill it with plane z + 3
            if (!__syncthreads_and(good)) return false;
            if (z + 3 <= ke + 1) issue(z + 3, s0);
            s0 = s1;
            return true;
        };

        for (int z = kb - 1; z <= ke; z += 2) {
            if (!step(z, kcA, rA, dA, kcB, rB, dB)) { ok = false; break; }
            if (z + 1 > ke) break;
            if (!step(z + 1, kcB, rB, dB, kcA, rA, dA)) { ok = false; break; }
        }
    }
    if (!ok) {
        // error path (a stage never arrived): wait, again with the limit, for the copies
        // still in flight into this CTA's shared memory before returning
        for (int s = 0; s < TB_NSTAGE; ++s)
            if (pend & (1u << s)) (void)wait(s);
    }
}

}  // namespace rfb
