// Host side of the C ABI declared in include/rfb_soc.h: device buffers, the solve driver
// (pseudo-time loop with periodic FP64 residual checks, FP32 defect correction), state
// management. All kernels live in soc_kernels.cuh.
#include "rfb_soc.h"
#include "soc_kernels.cuh"
#include "sweep_tb.cuh"
#include "sweep_dt.cuh"
#include "sweep_t3.cuh"
#include "bv_kernels.cuh"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

using namespace rfb;

namespace {

constexpr double R_GAS = 8.314462618;
constexpr double FARADAY = 96485.33212;

thread_local std::string g_create_error;

struct OpPoint {
    bool valid = false;
    double s_in = 0, eta = 0, beta = 1, cfl = 0.4;
    int inlet_bc = 0, dt_mode = 1, umt = 0;
    double A = 0, B = 0;      // affine rate law intercept / -slope
    double K1 = 0;            // e^{alpha eta~} - e^{(alpha-1) eta~} (kinetics mode 1)
    double dt = 0;            // global step
    double dmin = 0;          // smallest diagonal (local-dt bookkeeping)
};

}  // namespace

struct rfb_soc_handle {
    int nx = 0, ny = 0, nz = 0, nxny = 0;
    int64_t N = 0;
    double h = 0, D = 0;
    rfb_kinetics kin{};
    int device = 0;
    cudaStream_t stream = nullptr;

    unsigned char* d_arena = nullptr;   // one allocation holding the buffers below up to
                                        // d_partials (see rfb_soc_create)
    uint8_t* d_flags = nullptr;
    uint8_t* d_mask32 = nullptr;   // mask byte of the FP32 kernels
    double *d_u = nullptr, *d_v = nullptr, *d_w = nullptr;      // m/s, cell aligned
    double *d_us = nullptr, *d_vs = nullptr, *d_ws = nullptr;   // * beta / h
    float *d_u32 = nullptr, *d_v32 = nullptr, *d_w32 = nullptr; // * beta / h, FP32
    double* d_m = nullptr;
    float* d_m32 = nullptr;
    double* d_s[2] = {nullptr, nullptr};
    double* d_t[2] = {nullptr, nullptr};   // U_mt state
    float* d_delta[2] = {nullptr, nullptr};
    float* d_r32 = nullptr;
    float* d_dtc = nullptr;
    double* d_partials = nullptr;
    double* d_red = nullptr;
    double* h_red = nullptr;                // pinned, NRED doubles
    unsigned long long* d_err = nullptr;
    int s_cur = 0, t_cur = 0;
    bool have_state = false;
    bool have_umt_state = false;
    bool s_converged = false;     // state is a converged solve at op (adjoint precondition)
    bool t_converged = false;     // U_mt state converged at umt_op
    OpPoint umt_op;
    double* d_eta = nullptr;      // Nernst model: eta~ on electrode cells (first use)
    int* d_elec = nullptr;        // Nernst model: electrode-cell list (+ count at [N])
    bool have_eta = false;
    double* d_lam[2] = {nullptr, nullptr};   // adjoint state (allocated on first use)
    double* d_g = nullptr;
    double* d_grad = nullptr;
    // assembled FP64 operator (6 neighbour coefficients, diagonal, source) and its key
    double* d_L64 = nullptr;
    L64 K{};
    bool L64_valid = false;
    double L64_key[8] = {};
    int64_t area_version = 0;
    // double-float copies for the mixed-precision checks: the operator (same layout as
    // d_L64) and the state being corrected (ping-pong); allocated on the first mixed solve
    float2* d_L2F = nullptr;
    bool L2F_valid = false;
    float2* d_sdf[2] = {nullptr, nullptr};
    int df_cur = 0;
    float2* d_gdf = nullptr;      // adjoint source as pairs (mixed-precision adjoints)
    double scaled_beta = NAN;
    double* d_stage = nullptr;    // N doubles: host inputs of set_state / set_area_mult
                                  // (allocated on the first such call, then reused)
    // Butler-Volmer model (one allocation on first use): O, R, H ping-pong, phi, phi_old,
    // potential right-hand side, kappa_c, membrane kappa, CG r, z, p, q, 1/diag
    double* d_bv = nullptr;
    double* d_bvpart = nullptr;   // BV_NB x NRED partials + 16 CG scalars
    int bv_cur = 0;
    bool have_bv = false;

    int64_t n_fluid = 0, n_elec = 0;
    double sum_w_in = 0, sum_w_out = 0;     // unscaled sums of inlet / outlet W
    OpPoint op;
    int64_t launches = 0;
    std::string err;

    int kchunk = 8;
    dim3 grid, block;
    int64_t nblocks = 0;
    int vkchunk = 8;          // vectorised FP32 sweep (nx % 4 == 0)
    dim3 vgrid, vblock;
    // temporally blocked FP32 sweep (nx % 16 == 0, no area multiplier)
    int tb_mode = -1;         // -1 not chosen yet, 0 one-sweep kernel, 1 two-sweep passes
    // two launch shapes of the two-sweep pass (sweep_tb.cuh): 0 persistent (one CTA per
    // SM, equal shares of the tile-major plane space), 1 one (tile, z chunk) item per CTA
    // with the chunk count that wastes least of the last wave; the autotuner picks one
    struct TBLaunch {
        int lc = 0;           // planes per z chunk
        int64_t total = 0;    // tiles x chunks x lc
        int64_t per = 0;      // positions per CTA
        dim3 grid;
    } tb_launch[4];           // 2, 3: the same shapes for the three-sweep pass
    int tb_variant = -1;      // -1 not chosen yet; bit 0 the launch shape; step-field
                              // passes only: bit 1 one more TMA stage of delta (two-sweep:
                              // four instead of three; three-sweep: five instead of four),
                              // bit 2 three sweeps per pass instead of two
    bool tm_ready = false;
    CUtensorMap tm_delta[2], tm_r, tm_u, tm_v, tm_w, tm_f, tm_t;
    float* tm_delta_ptr[2] = {nullptr, nullptr};
    double tb_tuned_plain_ms = 0, tb_tuned_tb_ms = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

struct Fail {
    rfb_status st;
};

void set_err(rfb_soc_handle* h, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
}

#define CK(h, call)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_err((h), "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                    __FILE__, __LINE__);                                               \
            throw Fail{e_ == cudaErrorMemoryAllocation ? RFB_ERR_OOM : RFB_ERR_CUDA};  \
        }                                                                              \
    } while (0)

#define LAUNCHED(h)                                                                     \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            set_err((h), "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),   \
                    __FILE__, __LINE__);                                               \
            throw Fail{RFB_ERR_CUDA};                                                  \
        }                                                                              \
        ++(h)->launches;                                                               \
    } while (0)

// Device memory of the handles comes from a stream-ordered pool the library owns (one per
// device): a handle created after another was destroyed reuses its memory without a
// cudaMalloc / cudaFree, each of which synchronises the whole device. The pool keeps up to
// 16 GB of freed memory for reuse and returns the rest to the driver at the next
// synchronisation. Allocations are ordered on the handle's stream; every host call that
// hands a buffer to another stream synchronises the handle's stream first.
cudaMemPool_t handle_pool(rfb_soc_handle* h, bool renew = false) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(h->device);
    if (it != pools.end() && !renew) return it->second;
    if (it != pools.end()) pools.erase(it);   // lost with the context (a device reset)
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = h->device;
    cudaMemPool_t p = nullptr;
    CK(h, cudaMemPoolCreate(&p, &props));
    uint64_t keep = 16ull << 30;
    CK(h, cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[h->device] = p;
    return p;
}

// A new buffer is zero-filled: the kernels leave cells they never update at the value they
// find (the FP32 forcing of solid cells stays 0, and the correction sweeps multiply it by
// the zero step of those cells), and memory the pool hands out again holds old data.
void pool_alloc(rfb_soc_handle* h, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 1);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, handle_pool(h), h->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (e == cudaErrorMemoryAllocation) {
            set_err(h, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
            throw Fail{RFB_ERR_OOM};
        }
        // the pool no longer exists (the context was reset): a new one
        CK(h, cudaMallocFromPoolAsync(p, bytes, handle_pool(h, true), h->stream));
    }
    CK(h, cudaMemsetAsync(*p, 0, bytes, h->stream));
}

template <typename T>
void dalloc(rfb_soc_handle* h, T** p, size_t n) {
    pool_alloc(h, (void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

int flat_grid(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 32);
}

Lattice lattice(const rfb_soc_handle* h) {
    return Lattice{h->nx, h->ny, h->nz, h->nxny, h->d_flags, h->d_mask32};
}

void kinetics_AB(const rfb_kinetics& k, double eta, double* A, double* B, double* K1) {
    const double VT = R_GAS * k.T / FARADAY;
    const double Vt = k.n_e * (-eta) / VT;   // V~ (mode 0) = eta~ (mode 1), Eq. etat-def
    *A = std::exp(k.alpha * Vt);
    *B = *A * (1.0 + std::exp(-Vt));
    *K1 = *A - std::exp((k.alpha - 1.0) * Vt);
}

template <typename T>
Coef<T> make_coef(const rfb_soc_handle* h, const OpPoint& op, bool correction, bool local) {
    Coef<T> C{};
    if constexpr (sizeof(T) == 8) {
        C.u = h->d_us; C.v = h->d_vs; C.w = h->d_ws; C.m = h->d_m;
    } else {
        C.u = h->d_u32; C.v = h->d_v32; C.w = h->d_w32; C.m = h->d_m32;
    }
    C.dtc = local ? h->d_dtc : nullptr;
    C.s_in = correction ? T(0) : T(op.s_in);
    C.Dh = T(h->D / (h->h * h->h));
    C.gDh = T((op.inlet_bc == RFB_INLET_GHOST ? 1.0 : 2.0) * h->D / (h->h * h->h));
    C.dt = T(op.dt);
    const bool nl = h->kin.mode == RFB_KIN_UNIFORM_ETA && !op.umt && !correction;
    for (int n = 0; n < 8; ++n) {
        const double kap = op.umt ? 0.0 : h->kin.k0 * n / h->h;
        C.rA[n] = (correction || op.umt) ? T(0) : T(kap * (nl ? op.K1 : op.A));
        C.rB[n] = T(kap * op.B);
    }
    C.umt = op.umt;
    C.nl = nl ? 1 : 0;
    C.alpha = T(h->kin.alpha);
    return C;
}

void reduce_readback(rfb_soc_handle* h, int min_slot0) {
    finalize_kernel<<<1, 256, 0, h->stream>>>(h->d_partials, h->nblocks, h->d_red, min_slot0);
    LAUNCHED(h);
    CK(h, cudaMemcpyAsync(h->h_red, h->d_red, NRED * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
}

// Face velocities times beta / h (FP64 and FP32 copies) for the velocity scale beta;
// nothing is launched when they already hold that scale. Every kernel that builds
// coefficients reads these copies, so each entry point that evaluates an operating point
// calls this first (an intervening U_mt solve or adjoint may have used another scale).
void rescale_velocities(rfb_soc_handle* h, double beta) {
    if (h->scaled_beta == beta) return;
    const double sc = beta / h->h;
    const int64_t N = h->N;
    scale_kernel<<<flat_grid(N), 256, 0, h->stream>>>(h->d_u, h->d_us, h->d_u32, sc, N);
    LAUNCHED(h);
    scale_kernel<<<flat_grid(N), 256, 0, h->stream>>>(h->d_v, h->d_vs, h->d_v32, sc, N);
    LAUNCHED(h);
    scale_kernel<<<flat_grid(N + h->nxny), 256, 0, h->stream>>>(h->d_w, h->d_ws, h->d_w32,
                                                                sc, N + h->nxny);
    LAUNCHED(h);
    h->scaled_beta = beta;
}

// Prepare velocities, tables and dt for an operating point.
void prepare(rfb_soc_handle* h, OpPoint& op) {
    rescale_velocities(h, op.beta);
    kinetics_AB(h->kin, op.eta, &op.A, &op.B, &op.K1);
    Coef<double> C = make_coef<double>(h, op, false, false);
    const bool local = op.dt_mode == RFB_DT_LOCAL;
    diag_kernel<<<h->grid, h->block, 0, h->stream>>>(lattice(h), C, op.cfl,
                                                     local ? h->d_dtc : nullptr,
                                                     h->d_partials, h->kchunk);
    LAUNCHED(h);
    reduce_readback(h, 1);
    const double dmax = h->h_red[NRED - 1];
    op.dmin = h->h_red[0];
    op.dt = dmax > 0 ? op.cfl / dmax : 0.0;
    op.valid = true;
}

void fill_result(const rfb_soc_handle* h, const OpPoint& op, rfb_solve_result* r,
                 int64_t n_unknown, const double* sums = nullptr) {
    const double* v = sums ? sums : h->h_red;
    const double h3 = h->h * h->h * h->h;
    const double scale = h->kin.n_e * FARADAY * h->kin.c0 * h3;
    // Q = beta * sum_in W h^2 ; tau = V_f / Q = N_f h / (beta sum_in W)
    const double Q = op.beta * h->sum_w_in * h->h * h->h;
    const double tau = Q > 0 ? (double)h->n_fluid * h3 / Q
                             : std::pow(h->nz * h->h, 2) / h->D;
    r->residual = n_unknown > 0 ? tau * std::sqrt(v[0] / (double)n_unknown) : 0.0;
    r->I_tot = scale * v[1];
    r->F_in_adv = scale * v[3];
    r->F_in = scale * (v[2] + v[3]);
    r->F_out = scale * v[4];
    const double net = r->F_out - r->F_in;
    r->mass_balance_rel = r->I_tot != 0 ? std::fabs(r->I_tot - net) / std::fabs(r->I_tot)
                                        : std::fabs(net);
    const double denom = h->kin.n_e * FARADAY * h->kin.c0 * Q * (1.0 - op.s_in);
    r->U = denom != 0 ? r->I_tot / denom : NAN;
    r->outlet_mean = v[5] != 0 ? v[4] / v[5] : NAN;
    r->dt = op.dt;
    r->tau = tau;
    r->nonfinite = (int64_t)v[6];
}

// The assembled FP64 operator of the operating point op (U_mt or state of charge),
// rebuilt only when the operating point or the area multipliers changed.
void ensure_L64(rfb_soc_handle* h, const OpPoint& op) {
    if (!h->d_L64) dalloc(h, &h->d_L64, (size_t)8 * h->N);
    Coef<double> C = make_coef<double>(h, op, false, false);
    const double key[8] = {(double)op.umt, op.s_in,           op.A,
                           op.B,           op.beta,           (double)op.inlet_bc,
                           (double)h->area_version, C.nl ? 2.0 : 1.0};
    if (h->L64_valid && std::memcmp(key, h->L64_key, sizeof key) == 0) return;
    h->L2F_valid = false;
    for (int q = 0; q < 6; ++q) h->K.f[q] = h->d_L64 + (size_t)q * h->N;
    h->K.diag = h->d_L64 + (size_t)6 * h->N;
    h->K.b = h->d_L64 + (size_t)7 * h->N;
    if (C.nl) {   // mode 1: transport only; the kernels add the nonlinear source
        for (int n = 0; n < 8; ++n) C.rA[n] = C.rB[n] = 0.0;
        C.nl = 0;
    }
    assemble64_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(lattice(h), C, h->K);
    LAUNCHED(h);
    std::memcpy(h->L64_key, key, sizeof key);
    h->L64_valid = true;
}

// FP64 check of the state (s, or t for U_mt): defect, reductions and outputs.
void check(rfb_soc_handle* h, const OpPoint& op, bool umt) {
    double** buf = umt ? h->d_t : h->d_s;
    const int cur = umt ? h->t_cur : h->s_cur;
    ensure_L64(h, op);
    const Coef<double> C = make_coef<double>(h, op, false, false);
    check64c_kernel<false, false><<<h->grid, h->block, 0, h->stream>>>(
        lattice(h), C, h->K, buf[cur], nullptr, nullptr, nullptr, h->d_partials, h->kchunk);
    LAUNCHED(h);
    reduce_readback(h, 0);
}

// FP64 check that also writes the FP32 forcing (mixed precision near the double-float
// floor); fuse: the state is s + delta, written to the other buffer.
void check_forcing64(rfb_soc_handle* h, const OpPoint& op, bool umt, bool fuse) {
    double** buf = umt ? h->d_t : h->d_s;
    int& cur = umt ? h->t_cur : h->s_cur;
    ensure_L64(h, op);
    const Coef<double> C = make_coef<double>(h, op, false, false);
    if (fuse) {
        check64c_kernel<true, true><<<h->grid, h->block, 0, h->stream>>>(
            lattice(h), C, h->K, buf[cur], h->d_delta[0], buf[cur ^ 1], h->d_r32, h->d_partials,
            h->kchunk);
        LAUNCHED(h);
        cur ^= 1;
    } else {
        check64c_kernel<false, true><<<h->grid, h->block, 0, h->stream>>>(
            lattice(h), C, h->K, buf[cur], nullptr, nullptr, h->d_r32, h->d_partials, h->kchunk);
        LAUNCHED(h);
    }
    reduce_readback(h, 0);
}

// ---- mixed-precision checks in double-float (check_df_kernel)

void ensure_L2F(rfb_soc_handle* h, const OpPoint& op) {
    ensure_L64(h, op);
    if (h->L2F_valid) return;
    if (!h->d_L2F) dalloc(h, &h->d_L2F, (size_t)8 * h->N);
    split64_kernel<<<flat_grid(8 * h->N), 256, 0, h->stream>>>(h->d_L64, h->d_L2F, 8 * h->N);
    LAUNCHED(h);
    h->L2F_valid = true;
}

// state (s, or t for U_mt) -> its double-float copy
void df_begin(rfb_soc_handle* h, bool umt) {
    if (!h->d_sdf[0]) {
        dalloc(h, &h->d_sdf[0], h->N);
        dalloc(h, &h->d_sdf[1], h->N);
    }
    double** buf = umt ? h->d_t : h->d_s;
    const int cur = umt ? h->t_cur : h->s_cur;
    split64_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(buf[cur], h->d_sdf[0], h->N);
    LAUNCHED(h);
    h->df_cur = 0;
}

// double-float copy -> the FP64 state
void df_end(rfb_soc_handle* h, bool umt) {
    double** buf = umt ? h->d_t : h->d_s;
    const int cur = umt ? h->t_cur : h->s_cur;
    join64_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(h->d_sdf[h->df_cur], buf[cur], h->N);
    LAUNCHED(h);
}

// defect of the double-float state (fuse: of state + delta, which becomes the state);
// refreshes the FP32 forcing; reductions 0, 6, 7 only
void check_df(rfb_soc_handle* h, const OpPoint& op, bool umt, bool fuse) {
    ensure_L2F(h, op);
    const size_t N = h->N;
    L2F K;
    for (int q = 0; q < 6; ++q) K.f[q] = h->d_L2F + q * N;
    K.diag = h->d_L2F + 6 * N;
    K.b = h->d_L2F + 7 * N;
    const int cur = h->df_cur;
    if (fuse) {
        check_df_kernel<true><<<h->grid, h->block, 0, h->stream>>>(
            lattice(h), K, h->d_sdf[cur], h->d_delta[0], h->d_sdf[cur ^ 1], h->d_r32,
            h->d_partials, op.umt, h->kchunk);
        h->df_cur ^= 1;
    } else {
        check_df_kernel<false><<<h->grid, h->block, 0, h->stream>>>(
            lattice(h), K, h->d_sdf[cur], nullptr, nullptr, h->d_r32, h->d_partials, op.umt,
            h->kchunk);
    }
    LAUNCHED(h);
    reduce_readback(h, 0);
}

// n FP64 sweeps on s (or t for U_mt), ping-pong, with the assembled operator
void sweeps64(rfb_soc_handle* h, const OpPoint& op, bool umt, int64_t n) {
    double** buf = umt ? h->d_t : h->d_s;
    int& cur = umt ? h->t_cur : h->s_cur;
    ensure_L64(h, op);
    const float* dtc = op.dt_mode == RFB_DT_LOCAL ? h->d_dtc : nullptr;
    Lattice L = lattice(h);
    const Coef<double> C = make_coef<double>(h, op, false, false);
    for (int64_t q = 0; q < n; ++q) {
        if (C.nl)
            sweep64c_kernel<true><<<h->grid, h->block, 0, h->stream>>>(
                L, h->K, dtc, op.dt, buf[cur], buf[cur ^ 1], op.umt, h->kchunk, C, op.cfl);
        else
            sweep64c_kernel<false><<<h->grid, h->block, 0, h->stream>>>(
                L, h->K, dtc, op.dt, buf[cur], buf[cur ^ 1], op.umt, h->kchunk, C, op.cfl);
        LAUNCHED(h);
        cur ^= 1;
    }
}

// n FP32 correction sweeps delta <- delta + dt (L delta + r), starting from delta = 0.
// The result is left in d_delta[0].
// ---- temporally blocked FP32 passes (TMA tensor maps, see sweep_tb.cuh)

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Two-sweep passes: with local steps the step-field pass (sweep_dt.cuh; 16-byte FP32
// rows: nx % 4 == 0, any area multipliers, since they enter only through the step);
// with the global step the mask-byte pass (sweep_tb.cuh; 16-byte rows of the 8-bit mask,
// no area multiplier streamed).
bool tb_eligible(const rfb_soc_handle* h, bool local) {
    if (h->nz < 2) return false;
    return local ? (h->nx % 4) == 0 : ((h->nx % 16) == 0 && h->d_m32 == nullptr);
}

void tb_encode(rfb_soc_handle* h, CUtensorMap* m, CUtensorMapDataType t, size_t esize, void* ptr,
               int planes, int box_w) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        CK(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                               cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) {
            set_err(h, "cuTensorMapEncodeTiled is not available from the driver");
            throw Fail{RFB_ERR_CUDA};
        }
        fn = (EncodeTiledFn)p;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)h->nx, (cuuint64_t)h->ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)h->nx * esize, (cuuint64_t)h->nxny * esize};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)TB_BH, 1};
    // no L2 promotion: a box row is fetched at sector granularity (a 256-byte promotion
    // would pull whole 256-byte chunks for the halo columns at both ends of every row)
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, t, 3, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_err(h, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        throw Fail{RFB_ERR_CUDA};
    }
}

void tb_prepare(rfb_soc_handle* h) {
    if (h->tm_ready) return;
    // The shared-memory limit is an attribute of the kernel in the current device's
    // context, so it is set for every handle (with its device current): a process-wide
    // flag would leave a second device, or a context rebuilt after cudaDeviceReset, at
    // the default 48 KB and the launches would fail.
    {
        CK(h, cudaFuncSetAttribute(sweep32tb_kernel<false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, TB_SMEM));
        CK(h, cudaFuncSetAttribute(sweep32tb_kernel<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, TB_SMEM));
        CK(h, cudaFuncSetAttribute(sweep32tbd_kernel<false, 3>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tbd_smem<3>()));
        CK(h, cudaFuncSetAttribute(sweep32tbd_kernel<true, 3>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tbd_smem<3>()));
        CK(h, cudaFuncSetAttribute(sweep32tbd_kernel<false, 4>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tbd_smem<4>()));
        CK(h, cudaFuncSetAttribute(sweep32tbd_kernel<true, 4>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tbd_smem<4>()));
        CK(h, cudaFuncSetAttribute(sweep32t3_kernel<false, 4>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, t3_smem<4>()));
        CK(h, cudaFuncSetAttribute(sweep32t3_kernel<true, 4>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, t3_smem<4>()));
        CK(h, cudaFuncSetAttribute(sweep32t3_kernel<false, 5>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, t3_smem<5>()));
        CK(h, cudaFuncSetAttribute(sweep32t3_kernel<true, 5>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, t3_smem<5>()));
    }
    for (int q = 0; q < 2; ++q) {
        tb_encode(h, &h->tm_delta[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_delta[q], h->nz,
                  TB_BW);
        h->tm_delta_ptr[q] = h->d_delta[q];
    }
    tb_encode(h, &h->tm_r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_r32, h->nz, TB_BW);
    tb_encode(h, &h->tm_u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_u32, h->nz, TB_BW);
    tb_encode(h, &h->tm_v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_v32, h->nz, TB_BW);
    tb_encode(h, &h->tm_w, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_w32, h->nz + 1, TB_BW);
    if (h->nx % 16 == 0)   // the mask byte of the global-step pass
        tb_encode(h, &h->tm_f, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, h->d_mask32, h->nz, TB_BWM);
    tb_encode(h, &h->tm_t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_dtc, h->nz, TB_BW);
    // One CTA per SM fits (152 to 227 KB of shared memory each).
    // Shape 0, persistent: the tile-major (tile, plane) space in equal shares of at least
    // 16 planes (every z segment pays a prologue of k planes, k the sweeps of a pass): no
    // partial last wave, but CTAs on neighbouring tiles run at different planes and do not
    // share halo rows in L2.
    // Shape 1, chunked: one (tile, z chunk) item per CTA in chunk-major order, so that
    // neighbouring tiles run together; the chunk count minimises waves x (chunk + k).
    int sms = 152;
    CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    for (int k = 2; k <= 3; ++k) {
        const int rows = k == 2 ? TB_TYI : T3_TYI;
        const int64_t tiles = (int64_t)((h->nx + TB_TXI - 1) / TB_TXI) *
                              ((h->ny + rows - 1) / rows);
        auto& P = h->tb_launch[2 * (k - 2)];
        P.lc = h->nz;
        P.total = tiles * h->nz;
        P.per = std::max<int64_t>((P.total + sms - 1) / sms, 16);
        P.grid = dim3((unsigned)((P.total + P.per - 1) / P.per));
        int best_c = 1;
        double best = INFINITY;
        for (int c = 1; c <= std::max(1, h->nz / 8); ++c) {
            const int lc = (h->nz + c - 1) / c, cc = (h->nz + lc - 1) / lc;
            const double cost = std::ceil((double)(tiles * cc) / sms) * (lc + k);
            if (cost < best) { best = cost; best_c = cc; }
        }
        auto& Q = h->tb_launch[2 * (k - 2) + 1];
        Q.lc = (h->nz + best_c - 1) / best_c;
        Q.total = tiles * best_c * Q.lc;
        Q.per = Q.lc;
        Q.grid = dim3((unsigned)(tiles * best_c));
    }
    h->tm_ready = true;
}

unsigned int* tb_err_word(rfb_soc_handle* h) { return reinterpret_cast<unsigned int*>(h->d_err + 3); }

// sweeps of one pass of the chosen variant
int tb_depth(const rfb_soc_handle* h) { return h->tb_variant >= 4 ? 3 : 2; }

// one pass (two or three sweeps) from delta[cur] into delta[cur ^ 1] (tr: of the
// transposed operator; local steps only)
void tb_pass(rfb_soc_handle* h, const OpPoint& op, const Coef<float>& C, int cur, bool local,
             bool tr = false) {
    const CUtensorMap& td = (h->d_delta[cur] == h->tm_delta_ptr[0]) ? h->tm_delta[0]
                                                                     : h->tm_delta[1];
    if (local) {
        TBDArgs A{};
        A.nx = h->nx; A.ny = h->ny; A.nz = h->nz;
        const int v = std::max(h->tb_variant, 0);
        const auto& S = h->tb_launch[v >= 4 ? 2 + (v & 1) : v & 1];
        A.lc = S.lc; A.total = S.total; A.per = S.per;
        A.d_in = h->d_delta[cur];
        A.d_out = h->d_delta[cur ^ 1];
        A.omc = (float)(1.0 - op.cfl);
        A.Dh = C.Dh;
        A.err = tb_err_word(h);
        const bool four = (v & 2) != 0;
        if (v >= 4) {
            if (tr && four)
                sweep32t3_kernel<true, 5><<<S.grid, T3_THREADS, t3_smem<5>(), h->stream>>>(
                    td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
            else if (tr)
                sweep32t3_kernel<true, 4><<<S.grid, T3_THREADS, t3_smem<4>(), h->stream>>>(
                    td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
            else if (four)
                sweep32t3_kernel<false, 5><<<S.grid, T3_THREADS, t3_smem<5>(), h->stream>>>(
                    td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
            else
                sweep32t3_kernel<false, 4><<<S.grid, T3_THREADS, t3_smem<4>(), h->stream>>>(
                    td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
            LAUNCHED(h);
            return;
        }
        if (tr && four)
            sweep32tbd_kernel<true, 4><<<S.grid, TB_THREADS, tbd_smem<4>(), h->stream>>>(
                td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
        else if (tr)
            sweep32tbd_kernel<true, 3><<<S.grid, TB_THREADS, tbd_smem<3>(), h->stream>>>(
                td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
        else if (four)
            sweep32tbd_kernel<false, 4><<<S.grid, TB_THREADS, tbd_smem<4>(), h->stream>>>(
                td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
        else
            sweep32tbd_kernel<false, 3><<<S.grid, TB_THREADS, tbd_smem<3>(), h->stream>>>(
                td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_t, A);
        LAUNCHED(h);
        return;
    }
    TBArgs A{};
    A.nx = h->nx; A.ny = h->ny; A.nz = h->nz;
    const auto& S = h->tb_launch[std::max(h->tb_variant, 0) & 1];
    A.lc = S.lc; A.total = S.total; A.per = S.per;
    A.d_in = h->d_delta[cur];
    A.d_out = h->d_delta[cur ^ 1];
    A.Dh = C.Dh; A.gDh = C.gDh; A.dt = C.dt; A.cfl = (float)op.cfl; A.umt = C.umt;
    for (int q = 0; q < 8; ++q) A.tB[q] = C.rB[q];
    A.err = tb_err_word(h);
    if (local)
        sweep32tb_kernel<true><<<S.grid, TB_THREADS, TB_SMEM, h->stream>>>(
            td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_f, A);
    else
        sweep32tb_kernel<false><<<S.grid, TB_THREADS, TB_SMEM, h->stream>>>(
            td, h->tm_r, h->tm_u, h->tm_v, h->tm_w, h->tm_f, A);
    LAUNCHED(h);
}

DArgs dargs(const rfb_soc_handle* h, const OpPoint& op, const Coef<float>& C) {
    DArgs A{};
    A.nx = h->nx; A.ny = h->ny; A.nz = h->nz; A.nxny = h->nxny;
    A.u = h->d_u32; A.v = h->d_v32; A.w = h->d_w32; A.dt = h->d_dtc;
    A.omc = (float)(1.0 - op.cfl);
    A.Dh = C.Dh;
    return A;
}

// one plain sweep from delta[cur] into delta[cur ^ 1] (local steps: the step-field
// kernel, whose updates are bitwise those of the two-sweep pass)
void plain_sweep(rfb_soc_handle* h, const OpPoint& op, const Coef<float>& C, int cur,
                 bool local) {
    const bool vec = (h->nx % 4) == 0;
    Lattice L = lattice(h);
    if (vec && local)
        sweep32d_kernel<false><<<h->vgrid, h->vblock, 0, h->stream>>>(
            dargs(h, op, C), h->d_delta[cur], h->d_delta[cur ^ 1], h->d_r32, h->vkchunk);
    else if (vec)
        sweep32v_kernel<false><<<h->vgrid, h->vblock, 0, h->stream>>>(
            L, C, h->d_delta[cur], h->d_delta[cur ^ 1], h->d_r32, (float)op.cfl, h->vkchunk);
    else
        sweep_kernel<float, true><<<h->grid, h->block, 0, h->stream>>>(
            L, C, h->d_delta[cur], h->d_delta[cur ^ 1], h->d_r32, h->kchunk);
    LAUNCHED(h);
}

// n FP32 correction sweeps delta <- delta + dt (L delta + r), starting from delta = 0.
// The result is left in d_delta[0]. use_tb: passes of the chosen variant (two or three
// sweeps each), plain sweeps for the remainder.
void sweeps32(rfb_soc_handle* h, const OpPoint& op, int64_t n, bool use_tb = false) {
    const size_t bytes = (size_t)h->N * sizeof(float);
    CK(h, cudaMemsetAsync(h->d_delta[0], 0, bytes, h->stream));
    CK(h, cudaMemsetAsync(h->d_delta[1], 0, bytes, h->stream));
    const bool local = op.dt_mode == RFB_DT_LOCAL;
    const bool vec = (h->nx % 4) == 0;
    // the vectorised kernels compute the local step on the fly; the scalar one reads dtc
    Coef<float> C = make_coef<float>(h, op, true, local && !vec);
    int cur = 0;
    int64_t q = 0;
    if (use_tb) {
        tb_prepare(h);
        const int k = tb_depth(h);
        for (; q + k <= n; q += k) {
            tb_pass(h, op, C, cur, local);
            cur ^= 1;
        }
    }
    for (; q < n; ++q) {
        plain_sweep(h, op, C, cur, local);
        cur ^= 1;
    }
    if (cur == 1) {
        std::swap(h->d_delta[0], h->d_delta[1]);
        if (h->tm_ready) {
            std::swap(h->tm_delta[0], h->tm_delta[1]);
            std::swap(h->tm_delta_ptr[0], h->tm_delta_ptr[1]);
        }
    }
}

// n FP32 correction sweeps of the transposed operator (adjoint), delta <- delta +
// dt (L^T delta + r), from delta = 0; the result is left in d_delta[0] (nx % 4 == 0).
// With local steps: passes of the step-field kernels (two or three sweeps each, the
// variant the autotuner chose), plain sweeps for the remainder.
void sweeps32_adjoint(rfb_soc_handle* h, const OpPoint& op, const Coef<float>& C, int64_t n) {
    const size_t bytes = (size_t)h->N * sizeof(float);
    CK(h, cudaMemsetAsync(h->d_delta[0], 0, bytes, h->stream));
    CK(h, cudaMemsetAsync(h->d_delta[1], 0, bytes, h->stream));
    const bool local = op.dt_mode == RFB_DT_LOCAL;
    Lattice L = lattice(h);
    int cur = 0;
    int64_t q = 0;
    if (local && tb_eligible(h, true)) {
        tb_prepare(h);
        if (h->tb_variant < 0) h->tb_variant = 1;   // chunked shape unless tuned
        const int k = tb_depth(h);
        for (; q + k <= n; q += k) {
            tb_pass(h, op, C, cur, true, true);
            cur ^= 1;
        }
    }
    for (; q < n; ++q) {
        if (local)
            sweep32d_kernel<true><<<h->vgrid, h->vblock, 0, h->stream>>>(
                dargs(h, op, C), h->d_delta[cur], h->d_delta[cur ^ 1], h->d_r32, h->vkchunk);
        else
            sweep32v_kernel<false, true><<<h->vgrid, h->vblock, 0, h->stream>>>(
                L, C, h->d_delta[cur], h->d_delta[cur ^ 1], h->d_r32, (float)op.cfl, h->vkchunk);
        LAUNCHED(h);
        cur ^= 1;
    }
    if (cur == 1) {
        std::swap(h->d_delta[0], h->d_delta[1]);
        if (h->tm_ready) {
            std::swap(h->tm_delta[0], h->tm_delta[1]);
            std::swap(h->tm_delta_ptr[0], h->tm_delta_ptr[1]);
        }
    }
}

// Choices of the FP32-kernel autotuner, kept for the process by lattice shape (dims,
// area multipliers or not, dt mode, device): a new handle on the same shape reuses them.
struct TuneKey {
    int nx, ny, nz, mult, local, device;
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, nz, mult, local, device) <
               std::tie(o.nx, o.ny, o.nz, o.mult, o.local, o.device);
    }
};
struct TuneVal {
    int tb_mode, tb_variant;
    double plain_ms, tb_ms;
};
std::map<TuneKey, TuneVal> g_tune_cache;
std::mutex g_tune_mu;

// Project-written autotuner for one lattice: time (twice, keeping the faster) 12 plain
// sweeps and 12 sweeps of each
// launch shape of the two-sweep pass (with local steps: with three and with four TMA
// stages, and the three-sweep pass with four and five delta stages) by CUDA events on
// the current forcing and keep the fastest (tb_only: choose between the pass variants
// only).
void tune_fp32_kernel(rfb_soc_handle* h, const OpPoint& op, bool tb_only = false) {
    if (!tb_eligible(h, op.dt_mode == RFB_DT_LOCAL)) { h->tb_mode = 0; return; }
    const TuneKey key{h->nx, h->ny, h->nz, h->d_m32 != nullptr,
                      op.dt_mode == RFB_DT_LOCAL, h->device};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && (tb_only || it->second.tb_mode >= 0)) {
            h->tb_variant = it->second.tb_variant;
            if (!tb_only) h->tb_mode = it->second.tb_mode;
            h->tb_tuned_plain_ms = it->second.plain_ms;
            h->tb_tuned_tb_ms = it->second.tb_ms;
            return;
        }
    }
    // candidates: plain, then pass variants 0 .. nvar-1 (12 sweeps: whole passes of each)
    const int nvar = op.dt_mode == RFB_DT_LOCAL ? 8 : 2;
    float ms[9];
    for (float& m : ms) m = INFINITY;
    for (int cand = tb_only ? 1 : 0; cand <= nvar; ++cand) {
        if (cand > 0) h->tb_variant = cand - 1;
        sweeps32(h, op, 6, cand > 0);   // warm-up (and tensor maps)
        for (int rep = 0; rep < 2; ++rep) {   // the faster of two timings
            float t = 0.f;
            CK(h, cudaEventRecord(h->ev[0], h->stream));
            sweeps32(h, op, 12, cand > 0);
            CK(h, cudaEventRecord(h->ev[1], h->stream));
            CK(h, cudaEventSynchronize(h->ev[1]));
            CK(h, cudaEventElapsedTime(&t, h->ev[0], h->ev[1]));
            ms[cand] = std::min(ms[cand], t);
        }
    }
    int bestv = 0;
    for (int v = 1; v < nvar; ++v)
        if (ms[1 + v] < ms[1 + bestv]) bestv = v;
    h->tb_variant = bestv;
    const float tb = ms[1 + bestv];
    h->tb_tuned_plain_ms = ms[0] / 12;
    h->tb_tuned_tb_ms = tb / 12;
    if (!tb_only) h->tb_mode = tb < ms[0] ? 1 : 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TuneVal{tb_only ? -1 : h->tb_mode, h->tb_variant, h->tb_tuned_plain_ms,
                                h->tb_tuned_tb_ms};
}

void init_state(rfb_soc_handle* h, bool umt, double s_in) {
    double** buf = umt ? h->d_t : h->d_s;
    init_state_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(h->d_flags, buf[0], buf[1],
                                                              s_in, umt ? 1 : 0, h->N);
    LAUNCHED(h);
    if (umt) { h->t_cur = 0; h->have_umt_state = true; }
    else { h->s_cur = 0; h->have_state = true; }
}

bool read_opts(rfb_soc_handle* h, const rfb_solve_opts* in, rfb_solve_opts* o) {
    rfb_solve_opts_default(o);
    if (in) *o = *in;
    if (o->precision != RFB_PREC_FP64 && o->precision != RFB_PREC_MIXED) {
        set_err(h, "opts.precision must be RFB_PREC_FP64 or RFB_PREC_MIXED");
        return false;
    }
    if (o->inlet_bc != RFB_INLET_FACE && o->inlet_bc != RFB_INLET_GHOST) {
        set_err(h, "opts.inlet_bc invalid");
        return false;
    }
    if (o->dt_mode != RFB_DT_GLOBAL && o->dt_mode != RFB_DT_LOCAL) {
        set_err(h, "opts.dt_mode invalid");
        return false;
    }
    if (!(o->cfl > 0 && o->cfl <= 1.0)) { set_err(h, "opts.cfl must be in (0, 1]"); return false; }
    if (!(o->velocity_scale >= 0 && std::isfinite(o->velocity_scale))) {
        set_err(h, "opts.velocity_scale must be finite and >= 0");
        return false;
    }
    if (o->check_every < 0 || o->max_sweeps < 0) {
        set_err(h, "opts.check_every / max_sweeps must be >= 0");
        return false;
    }
    for (int q = 0; q < 6; ++q)
        if (o->reserved[q] != 0) { set_err(h, "opts.reserved must be zero"); return false; }
    if (o->timeout_ms < 0) { set_err(h, "opts.timeout_ms must be >= 0"); return false; }
    if (o->fp32_kernel < 0 || o->fp32_kernel > 10 ||
        (o->fp32_kernel >= 5 && o->dt_mode != RFB_DT_LOCAL)) {
        set_err(h, "opts.fp32_kernel must be 0 (auto), 1 (one sweep), 2 (passes), 3 / 4 "
                   "(two-sweep passes, persistent / chunked launch) or, with local steps, "
                   "5 / 6 (the same with four TMA stages), 7 / 8 (three-sweep passes) or "
                   "9 / 10 (three-sweep passes with five delta stages)");
        return false;
    }
    if (o->fp32_kernel >= 2 && !tb_eligible(h, o->dt_mode == RFB_DT_LOCAL)) {
        set_err(h, "two-sweep passes need nz >= 2 and nx %% 4 == 0 (local steps), or nx %% 16 "
                   "== 0 and no area multiplier (global step)");
        return false;
    }
    if (o->max_sweeps == 0) o->max_sweeps = 50000000;
    return true;
}

OpPoint make_op(const rfb_solve_opts& o, double s_in, double eta, bool umt) {
    OpPoint op;
    op.s_in = umt ? 0.0 : s_in;
    op.eta = eta;
    op.beta = o.velocity_scale;
    op.cfl = o.cfl;
    op.inlet_bc = o.inlet_bc;
    op.dt_mode = o.dt_mode;
    op.umt = umt ? 1 : 0;
    return op;
}

int64_t default_check_every(const rfb_soc_handle* h, int precision) {
    // one FP64 check per ~this many sweeps: cheap for small lattices (launch bound),
    // negligible for large ones
    (void)h;
    return precision == RFB_PREC_MIXED ? 200 : 100;
}

// Core driver shared by solve / step / umt. Returns the status; fills res.
rfb_status drive(rfb_soc_handle* h, const rfb_solve_opts& o, OpPoint& op, bool umt,
                 double tol, int64_t fixed_sweeps, rfb_solve_result* res) {
    auto t0 = std::chrono::steady_clock::now();
    prepare(h, op);
    const int64_t n_unknown = umt ? h->n_fluid - h->n_elec : h->n_fluid;
    bool& have = umt ? h->have_umt_state : h->have_state;
    if (!have) init_state(h, umt, op.s_in);
    const bool mixed = o.precision == RFB_PREC_MIXED;
    if (mixed && !umt && h->kin.mode != RFB_KIN_AFFINE) {
        set_err(h, "kinetics mode 1 (nonlinear source) runs in RFB_PREC_FP64 only");
        throw Fail{RFB_ERR_INVALID_ARG};
    }
    int64_t every = o.check_every > 0 ? o.check_every : default_check_every(h, o.precision);
    rfb_solve_result r{};
    rfb_status st = RFB_OK;
    int64_t done = 0;
    double sweep_ms = 0.0, check_ms = 0.0;
    const int64_t limit = fixed_sweeps >= 0 ? fixed_sweeps : o.max_sweeps;
    // first check: residual of the starting state (mixed: of its double-float copy, and
    // the FP32 forcing)
    if (mixed) {
        df_begin(h, umt);
        check_df(h, op, umt, false);
    } else {
        check(h, op, umt);
    }
    ++r.checks;
    fill_result(h, op, &r, n_unknown);
    // mixed: the FP64 state equals the double-float one and r holds its FP64 check
    bool joined = !mixed;
    // mixed: defects in double-float until the residual nears that arithmetic's floor,
    // about tau 2^-47 (8 terms of size <= max d_c, s <= 1); FP64 defects after that
    bool df = mixed;
    const double df_floor = mixed ? r.tau * std::ldexp(1.0, -44) * (op.cfl / op.dt) : 0.0;
    auto join_and_check = [&]() {
        CK(h, cudaEventRecord(h->ev[1], h->stream));
        df_end(h, umt);
        check(h, op, umt);
        CK(h, cudaEventRecord(h->ev[2], h->stream));
        CK(h, cudaEventSynchronize(h->ev[2]));
        float ms_c = 0.f;
        CK(h, cudaEventElapsedTime(&ms_c, h->ev[1], h->ev[2]));
        check_ms += ms_c;
        ++r.checks;
        fill_result(h, op, &r, n_unknown);
        joined = true;
    };
    // FP32 kernel: one-sweep or two-sweep passes (forced by opts or autotuned once)
    bool use_tb = false;
    if (mixed) {
        if (o.fp32_kernel == 2) {
            if (h->tb_variant < 0) tune_fp32_kernel(h, op, true);
            use_tb = true;
        } else if (o.fp32_kernel >= 3) {
            // a forced variant (kept for later calls): 3 / 4 and 5 / 6 two-sweep passes with
            // three / four TMA stages, 7 / 8 and 9 / 10 three-sweep passes with four / five
            h->tb_variant = o.fp32_kernel <= 4 ? o.fp32_kernel - 3
                            : o.fp32_kernel <= 6 ? (o.fp32_kernel - 5) | 2
                            : o.fp32_kernel <= 8 ? (o.fp32_kernel - 7) | 4
                                                  : (o.fp32_kernel - 9) | 6;
            use_tb = true;
        } else if (o.fp32_kernel == 0) {
            if (h->tb_mode < 0) tune_fp32_kernel(h, op);
            use_tb = h->tb_mode == 1;
        }
        if (use_tb) CK(h, cudaMemsetAsync(tb_err_word(h), 0, sizeof(unsigned int), h->stream));
    }
    // sweeps per pass: the default interval and the shortened ones are whole passes
    const int depth = use_tb ? tb_depth(h) : 1;
    if (o.check_every == 0) every = std::max<int64_t>(depth, every / depth * depth);
    // Check interval: `every` sweeps, shortened near the end. The residual of these
    // transport problems does not decay geometrically early on (it stays up while the
    // inlet state is carried through the lattice, then falls faster), so a crossing
    // extrapolated from the last two checks lies too late there and the interval stays at
    // `every`; in the geometric tail the extrapolation is accurate, and the next check is
    // placed just past the predicted crossing of tol (at least 16 sweeps, whole passes) instead of
    // up to `every` sweeps beyond it; intervals are whole passes of the FP32 kernel. One
    // check costs about 9 to 13 FP32 sweeps.
    int64_t next_every = every;
    while (true) {
        if (r.nonfinite > 0) { st = RFB_ERR_NONFINITE; break; }
        if (fixed_sweeps < 0 && r.residual <= tol) {
            if (joined) break;
            join_and_check();   // the double-float defect met tol: confirm it in FP64
            continue;
        }
        if (df && fixed_sweeps < 0 && r.residual <= 10.0 * df_floor) {
            // tol lies below what double-float defects resolve: continue with FP64 ones
            df_end(h, umt);
            CK(h, cudaEventRecord(h->ev[1], h->stream));
            check_forcing64(h, op, umt, false);
            CK(h, cudaEventRecord(h->ev[2], h->stream));
            CK(h, cudaEventSynchronize(h->ev[2]));
            float ms_c = 0.f;
            CK(h, cudaEventElapsedTime(&ms_c, h->ev[1], h->ev[2]));
            check_ms += ms_c;
            ++r.checks;
            fill_result(h, op, &r, n_unknown);
            df = false;
            joined = true;
            continue;
        }
        if (done >= limit) {
            st = fixed_sweeps >= 0 ? RFB_OK : RFB_ERR_NOT_CONVERGED;
            break;
        }
        if (o.timeout_ms > 0 &&
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count() >= o.timeout_ms) {
            set_err(h, "opts.timeout_ms reached after %lld sweeps", (long long)done);
            st = RFB_ERR_NOT_CONVERGED;
            break;
        }
        const int64_t n = std::min(next_every, limit - done);
        CK(h, cudaEventRecord(h->ev[0], h->stream));
        if (mixed) sweeps32(h, op, n, use_tb);
        else sweeps64(h, op, umt, n);
        CK(h, cudaEventRecord(h->ev[1], h->stream));
        if (df) {
            check_df(h, op, umt, true);
            joined = false;
        } else if (mixed) {
            check_forcing64(h, op, umt, true);   // FP64 defects (below the df floor)
        } else {
            check(h, op, umt);
        }
        CK(h, cudaEventRecord(h->ev[2], h->stream));   // check() synchronised the stream
        CK(h, cudaEventSynchronize(h->ev[2]));
        float ms_s = 0.f, ms_c = 0.f;
        CK(h, cudaEventElapsedTime(&ms_s, h->ev[0], h->ev[1]));
        CK(h, cudaEventElapsedTime(&ms_c, h->ev[1], h->ev[2]));
        sweep_ms += ms_s;
        check_ms += ms_c;
        const double res_before = r.residual;
        done += n;
        ++r.checks;
        fill_result(h, op, &r, n_unknown);
        next_every = every;
        if (fixed_sweeps < 0 && done > n && r.residual > tol && r.residual < res_before) {
            const double rate = std::log(res_before / r.residual) / (double)n;   // per sweep
            const double need = std::log(r.residual / tol) / rate;
            int64_t k = (int64_t)std::ceil(1.1 * need) + 2;
            k = std::max<int64_t>(16, k);
            k = (k + depth - 1) / depth * depth;
            next_every = std::min(every, k);
        }
    }
    if (!joined) {
        const rfb_status keep = st;
        join_and_check();   // the state and the outputs of the call in FP64
        if (keep == RFB_OK && r.nonfinite > 0) st = RFB_ERR_NONFINITE;
    }
    r.sweeps = done;
    r.sweep_ms = sweep_ms;
    r.check_ms = check_ms;
    r.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                    .count();
    if (use_tb) {
        unsigned int bad = 0;
        CK(h, cudaMemcpyAsync(&bad, tb_err_word(h), sizeof bad, cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (bad) {
            set_err(h, "a TMA stage of the two-sweep kernel did not arrive in time");
            st = RFB_ERR_CUDA;
        }
    }
    if (res) *res = r;
    return st;
}

rfb_status guard(rfb_soc_handle* h) {
    if (!h) return RFB_ERR_INVALID_ARG;
    (void)cudaGetLastError();   // drop a stale error left by an earlier failed runtime call
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        set_err(h, "cudaSetDevice: %s", cudaGetErrorString(e));
        return RFB_ERR_CUDA;
    }
    h->err.clear();
    return RFB_OK;
}

void free_all(rfb_soc_handle* h) {
    // the arena holds flags .. partials; the rest are allocated on first use
    void* ptrs[] = {h->d_arena, h->d_m,    h->d_m32,  h->d_lam[0], h->d_lam[1], h->d_g,
                    h->d_grad,  h->d_L64,  h->d_L2F,  h->d_eta,    h->d_elec,   h->d_sdf[0],
                    h->d_sdf[1], h->d_gdf,  h->d_stage,  h->d_bv,     h->d_bvpart};
    for (void* p : ptrs)   // back to the pool, in the handle's stream order
        if (p) cudaFreeAsync(p, h->stream);
    cudaStreamSynchronize(h->stream);
    if (h->h_red) cudaFreeHost(h->h_red);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

void rfb_solve_opts_default(rfb_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = RFB_PREC_FP64;
    o->inlet_bc = RFB_INLET_FACE;
    o->dt_mode = RFB_DT_LOCAL;
    o->check_every = 0;
    o->cfl = 0.4;
    o->velocity_scale = 1.0;
    o->max_sweeps = 0;
}

const char* rfb_status_string(rfb_status st) {
    switch (st) {
        case RFB_OK: return "ok";
        case RFB_ERR_INVALID_ARG: return "invalid argument";
        case RFB_ERR_CUDA: return "CUDA error";
        case RFB_ERR_OOM: return "out of device memory";
        case RFB_ERR_NOT_CONVERGED: return "not converged (state valid)";
        case RFB_ERR_NONFINITE: return "non-finite value in state or residual";
        case RFB_ERR_STATE: return "required state missing";
        case RFB_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char* rfb_soc_last_error(const rfb_soc_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

rfb_status rfb_soc_create(const int32_t dims[3], double dx, const uint8_t* fiber_mask,
                          const double* U, const double* V, const double* W, double D,
                          const rfb_kinetics* kin, const double* area_mult,
                          rfb_mem_kind kind, void* cuda_stream, rfb_soc_handle** out) {
    g_create_error.clear();
    if (!out) { set_err(nullptr, "out is NULL"); return RFB_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!dims || !fiber_mask || !U || !V || !W || !kin) {
        set_err(nullptr, "NULL input pointer");
        return RFB_ERR_INVALID_ARG;
    }
    if (kind != RFB_MEM_HOST && kind != RFB_MEM_DEVICE) {
        set_err(nullptr, "kind must be RFB_MEM_HOST or RFB_MEM_DEVICE");
        return RFB_ERR_INVALID_ARG;
    }
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    if (nx < 1 || ny < 1 || nz < 2) {
        set_err(nullptr, "dims must be >= (1, 1, 2)");
        return RFB_ERR_INVALID_ARG;
    }
    const int64_t N = (int64_t)nx * ny * nz;
    if (N + (int64_t)nx * ny >= ((int64_t)1 << 31)) {
        set_err(nullptr, "lattice too large: N + nx*ny must be < 2^31");
        return RFB_ERR_INVALID_ARG;
    }
    if (!(dx > 0 && std::isfinite(dx)) || !(D > 0 && std::isfinite(D))) {
        set_err(nullptr, "dx and D must be finite and > 0");
        return RFB_ERR_INVALID_ARG;
    }
    if (!(kin->k0 >= 0 && std::isfinite(kin->k0)) || !(kin->alpha > 0 && kin->alpha < 1) ||
        kin->n_e < 1 || !(kin->T > 0 && std::isfinite(kin->T)) ||
        !(kin->c0 > 0 && std::isfinite(kin->c0))) {
        set_err(nullptr, "kinetics out of range (k0 >= 0, 0 < alpha < 1, n_e >= 1, T > 0, c0 > 0)");
        return RFB_ERR_INVALID_ARG;
    }
    if (kin->mode != RFB_KIN_AFFINE && kin->mode != RFB_KIN_UNIFORM_ETA) {
        set_err(nullptr, "kinetics mode must be RFB_KIN_AFFINE (0) or RFB_KIN_UNIFORM_ETA (1)");
        return RFB_ERR_INVALID_ARG;
    }
    rfb_soc_handle* h = new rfb_soc_handle();
    try {
        h->nx = nx; h->ny = ny; h->nz = nz; h->nxny = nx * ny; h->N = N;
        h->h = dx; h->D = D; h->kin = *kin;
        h->stream = (cudaStream_t)cuda_stream;
        CK(h, cudaGetDevice(&h->device));
        const int64_t nxny = h->nxny;
        const int64_t nU = (int64_t)(nx + 1) * ny * nz, nV = (int64_t)nx * (ny + 1) * nz,
                      nW = nxny * (nz + 1);
        // launch geometry: 32 x 8 column tiles, z chunks so that there are >= ~8 blocks
        // per SM
        h->block = dim3(BX, BY, 1);
        const int gx = (nx + BX - 1) / BX, gy = (ny + BY - 1) / BY;
        int kc = nz;
        while (kc > 4 && (int64_t)gx * gy * ((nz + kc - 1) / kc) < 152 * 8) kc = (kc + 1) / 2;
        h->kchunk = kc;
        h->grid = dim3(gx, gy, (nz + kc - 1) / kc);
        h->nblocks = (int64_t)h->grid.x * h->grid.y * h->grid.z;
        {
            h->vblock = dim3(VBX, VBY, 1);
            const int vx = (nx / 4 + VBX - 1) / VBX, vy = (ny + VBY - 1) / VBY;
            int vk = nz;
            while (vk > 4 && (int64_t)vx * vy * ((nz + vk - 1) / vk) < 152 * 16) vk = (vk + 1) / 2;
            h->vkchunk = vk;
            h->vgrid = dim3(vx, vy, (nz + vk - 1) / vk);
        }
        // every buffer a handle always needs, carved from one device allocation (one
        // cudaMalloc / cudaFree per handle instead of ~25); sub-buffers 256-byte aligned
        {
            struct Part { void** p; size_t bytes; };
            const size_t n8 = (size_t)N * 8, n4 = (size_t)N * 4, nw8 = (size_t)(N + nxny) * 8,
                         nw4 = (size_t)(N + nxny) * 4;
            const Part parts[] = {
                {(void**)&h->d_flags, (size_t)N}, {(void**)&h->d_mask32, (size_t)N},
                {(void**)&h->d_u, n8}, {(void**)&h->d_v, n8}, {(void**)&h->d_w, nw8},
                {(void**)&h->d_us, n8}, {(void**)&h->d_vs, n8}, {(void**)&h->d_ws, nw8},
                {(void**)&h->d_u32, n4}, {(void**)&h->d_v32, n4}, {(void**)&h->d_w32, nw4},
                {(void**)&h->d_s[0], n8}, {(void**)&h->d_s[1], n8},
                {(void**)&h->d_t[0], n8}, {(void**)&h->d_t[1], n8},
                {(void**)&h->d_delta[0], n4}, {(void**)&h->d_delta[1], n4},
                {(void**)&h->d_r32, n4}, {(void**)&h->d_dtc, n4},
                {(void**)&h->d_err, 4 * sizeof(unsigned long long)},
                {(void**)&h->d_red, NRED * sizeof(double)},
                {(void**)&h->d_partials, (size_t)h->nblocks * NRED * sizeof(double)}};
            auto up = [](size_t b) { return (b + 255) / 256 * 256; };
            size_t total = 0;
            for (const Part& q : parts) total += up(q.bytes);
            pool_alloc(h, (void**)&h->d_arena, total);
            size_t off = 0;
            for (const Part& q : parts) {
                *q.p = h->d_arena + off;
                off += up(q.bytes);
            }
        }
        CK(h, cudaMallocHost((void**)&h->h_red, NRED * sizeof(double)));
        for (cudaEvent_t& e : h->ev) CK(h, cudaEventCreate(&e));

        // staging: the inputs on the device (copied when they are host arrays)
        uint8_t* d_mask = nullptr;
        double *dU = nullptr, *dV = nullptr, *dW = nullptr, *dm = nullptr;
        std::vector<void*> tmp;
        auto stage = [&](const void* src, size_t bytes, void** dst) {
            if (kind == RFB_MEM_DEVICE) { *dst = const_cast<void*>(src); return; }
            pool_alloc(h, dst, bytes);
            tmp.push_back(*dst);
            CK(h, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
        };
        try {
            stage(fiber_mask, N, (void**)&d_mask);
            stage(U, nU * 8, (void**)&dU);
            stage(V, nV * 8, (void**)&dV);
            stage(W, nW * 8, (void**)&dW);
            if (area_mult) stage(area_mult, N * 8, (void**)&dm);
            CK(h, cudaMemsetAsync(h->d_err, 0, 4 * sizeof(unsigned long long), h->stream));
            CK(h, cudaMemsetAsync(h->d_u, 0, N * 8, h->stream));
            CK(h, cudaMemsetAsync(h->d_v, 0, N * 8, h->stream));
            flags_kernel<<<flat_grid(N), 256, 0, h->stream>>>(d_mask, h->d_flags, h->d_mask32,
                                                              nx, ny, nz);
            LAUNCHED(h);
            repack_kernel<<<flat_grid(nU), 256, 0, h->stream>>>(dU, d_mask, h->d_u, nx, ny, nz,
                                                                0, h->d_err);
            LAUNCHED(h);
            repack_kernel<<<flat_grid(nV), 256, 0, h->stream>>>(dV, d_mask, h->d_v, nx, ny, nz,
                                                                1, h->d_err);
            LAUNCHED(h);
            repack_kernel<<<flat_grid(nW), 256, 0, h->stream>>>(dW, d_mask, h->d_w, nx, ny, nz,
                                                                2, h->d_err);
            LAUNCHED(h);
            if (area_mult) {
                dalloc(h, &h->d_m, N);
                dalloc(h, &h->d_m32, N);
                scale_kernel<<<flat_grid(N), 256, 0, h->stream>>>(dm, h->d_m, h->d_m32, 1.0, N);
                LAUNCHED(h);
            }
            // counts and inlet / outlet sums on the device (fixed-order reduction)
            const int sblocks = (int)std::min<int64_t>(h->nblocks, 2048);
            stats_kernel<<<sblocks, 256, 0, h->stream>>>(h->d_flags, h->d_w, h->d_m, N, nxny,
                                                         h->d_partials);
            LAUNCHED(h);
            finalize_kernel<<<1, 256, 0, h->stream>>>(h->d_partials, sblocks, h->d_red, 0);
            LAUNCHED(h);
            unsigned long long herr[4];
            CK(h, cudaMemcpyAsync(herr, h->d_err, sizeof herr, cudaMemcpyDeviceToHost,
                                  h->stream));
            CK(h, cudaMemcpyAsync(h->h_red, h->d_red, NRED * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            for (void* p : tmp) cudaFreeAsync(p, h->stream);
            tmp.clear();
            if (herr[0]) { set_err(nullptr, "%llu non-finite face velocities", herr[0]); throw Fail{RFB_ERR_INVALID_ARG}; }
            if (herr[1]) { set_err(nullptr, "%llu nonzero velocities on side-wall or fiber faces", herr[1]); throw Fail{RFB_ERR_INVALID_ARG}; }
            if (herr[2]) { set_err(nullptr, "%llu negative inlet/outlet velocities", herr[2]); throw Fail{RFB_ERR_INVALID_ARG}; }
            h->n_fluid = (int64_t)h->h_red[0];
            h->n_elec = (int64_t)h->h_red[1];
            h->sum_w_in = h->h_red[2];
            h->sum_w_out = h->h_red[3];
            if (h->h_red[4] > 0) {
                set_err(nullptr, "area_mult must be finite and > 0 (%.0f cells are not)", h->h_red[4]);
                throw Fail{RFB_ERR_INVALID_ARG};
            }
            if (h->n_fluid == 0) { set_err(nullptr, "no fluid cells"); throw Fail{RFB_ERR_INVALID_ARG}; }
        } catch (...) {
            cudaStreamSynchronize(h->stream);
            for (void* p : tmp) cudaFreeAsync(p, h->stream);
            throw;
        }
    } catch (Fail f) {
        if (!h->err.empty()) g_create_error = h->err;
        free_all(h);
        delete h;
        return f.st;
    }
    *out = h;
    return RFB_OK;
}

rfb_status rfb_soc_destroy(rfb_soc_handle* h) {
    if (!h) return RFB_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return RFB_OK;
}

rfb_status rfb_soc_set_stream(rfb_soc_handle* h, void* s) {
    rfb_status g = guard(h);
    if (g) return g;
    h->stream = (cudaStream_t)s;
    return RFB_OK;
}

rfb_status rfb_soc_solve(rfb_soc_handle* h, double s_in, double eta, double tol,
                         const rfb_solve_opts* opts, rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    rfb_solve_opts o;
    if (!read_opts(h, opts, &o)) return RFB_ERR_INVALID_ARG;
    if (!(s_in >= 0 && s_in <= 1)) { set_err(h, "s_in must be in [0, 1]"); return RFB_ERR_INVALID_ARG; }
    if (!std::isfinite(eta)) { set_err(h, "eta must be finite"); return RFB_ERR_INVALID_ARG; }
    if (!(tol > 0)) { set_err(h, "tol must be > 0"); return RFB_ERR_INVALID_ARG; }
    try {
        OpPoint op = make_op(o, s_in, eta, false);
        rfb_status st = drive(h, o, op, false, tol, -1, res);
        h->op = op;
        h->s_converged = (st == RFB_OK);
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_step(rfb_soc_handle* h, double s_in, double eta, int64_t n_sweeps,
                        const rfb_solve_opts* opts, rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    rfb_solve_opts o;
    if (!read_opts(h, opts, &o)) return RFB_ERR_INVALID_ARG;
    if (!(s_in >= 0 && s_in <= 1)) { set_err(h, "s_in must be in [0, 1]"); return RFB_ERR_INVALID_ARG; }
    if (!std::isfinite(eta)) { set_err(h, "eta must be finite"); return RFB_ERR_INVALID_ARG; }
    if (n_sweeps < 0) { set_err(h, "n_sweeps must be >= 0"); return RFB_ERR_INVALID_ARG; }
    try {
        OpPoint op = make_op(o, s_in, eta, false);
        if (o.check_every == 0) o.check_every = (int32_t)std::min<int64_t>(std::max<int64_t>(n_sweeps, 1), 1 << 30);
        h->s_converged = false;
        rfb_status st = drive(h, o, op, false, 0.0, n_sweeps, res);
        h->op = op;
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_current(rfb_soc_handle* h, rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    if (!h->have_state || !h->op.valid) {
        set_err(h, "no state / operating point: call rfb_soc_solve or rfb_soc_step first");
        return RFB_ERR_STATE;
    }
    try {
        OpPoint op = h->op;
        rescale_velocities(h, op.beta);
        check(h, op, false);
        rfb_solve_result r{};
        r.checks = 1;
        fill_result(h, op, &r, h->n_fluid);
        if (res) *res = r;
        return r.nonfinite ? RFB_ERR_NONFINITE : RFB_OK;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_umt(rfb_soc_handle* h, double tol, const rfb_solve_opts* opts, double* umt,
                       rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    rfb_solve_opts o;
    if (!read_opts(h, opts, &o)) return RFB_ERR_INVALID_ARG;
    if (!(tol > 0)) { set_err(h, "tol must be > 0"); return RFB_ERR_INVALID_ARG; }
    try {
        OpPoint op = make_op(o, 0.0, 0.0, true);
        h->have_umt_state = false;   // always a cold start: s = 0, electrode cells = 1
        rfb_solve_result r{};
        rfb_status st = drive(h, o, op, true, tol, -1, &r);
        h->umt_op = op;
        h->t_converged = (st == RFB_OK);
        if (umt) *umt = r.outlet_mean;
        if (res) *res = r;
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_solve_nernst(rfb_soc_handle* h, double s_in, double eta, double tol,
                                double omega, const rfb_solve_opts* opts,
                                rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    rfb_solve_opts o;
    if (!read_opts(h, opts, &o)) return RFB_ERR_INVALID_ARG;
    if (!(s_in >= 0 && s_in <= 1)) { set_err(h, "s_in must be in [0, 1]"); return RFB_ERR_INVALID_ARG; }
    if (!std::isfinite(eta)) { set_err(h, "eta must be finite"); return RFB_ERR_INVALID_ARG; }
    if (!(tol > 0)) { set_err(h, "tol must be > 0"); return RFB_ERR_INVALID_ARG; }
    if (!(omega > 0 && omega <= 1)) { set_err(h, "omega must be in (0, 1]"); return RFB_ERR_INVALID_ARG; }
    if (o.precision != RFB_PREC_FP64 || h->kin.mode != RFB_KIN_AFFINE || h->kin.alpha != 0.5 ||
        !(h->kin.k0 > 0)) {
        set_err(h, "the Nernst model needs RFB_PREC_FP64, kinetics mode 0, alpha = 1/2, k0 > 0");
        return RFB_ERR_INVALID_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    try {
        OpPoint op = make_op(o, s_in, eta, false);
        prepare(h, op);
        const int64_t N = h->N;
        if (!h->d_eta) dalloc(h, &h->d_eta, N);
        const bool warm = h->have_state;
        if (!warm) init_state(h, false, op.s_in);
        const Coef<double> C = make_coef<double>(h, op, false, false);
        const double kap0 = h->kin.k0 / h->h;
        const double Vt = h->kin.n_e * (-eta) / (R_GAS * h->kin.T / FARADAY);
        nernst_init_kernel<<<flat_grid(N), 256, 0, h->stream>>>(
            lattice(h), C, h->d_s[h->s_cur], h->d_s[h->s_cur ^ 1], h->d_eta, kap0, Vt,
            warm ? 1 : 0);
        LAUNCHED(h);
        h->have_eta = true;
        // the electrode cells as a list: their update runs in full warps of its own
        if (!h->d_elec) dalloc(h, &h->d_elec, N + 1);
        CK(h, cudaMemsetAsync(h->d_elec + N, 0, sizeof(int), h->stream));
        nernst_list_kernel<<<flat_grid(N), 256, 0, h->stream>>>(lattice(h), C, kap0, h->d_elec,
                                                                h->d_elec + N);
        LAUNCHED(h);
        int n_elec = 0;
        CK(h, cudaMemcpyAsync(&n_elec, h->d_elec + N, sizeof(int), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        ensure_L64(h, op);
        const float* dtc = op.dt_mode == RFB_DT_LOCAL ? h->d_dtc : nullptr;
        const int64_t every = o.check_every > 0 ? o.check_every : default_check_every(h, RFB_PREC_FP64);
        rfb_solve_result r{};
        rfb_status st = RFB_OK;
        int64_t done = 0;
        double sweep_ms = 0.0, check_ms = 0.0;
        check(h, op, false);
        ++r.checks;
        fill_result(h, op, &r, h->n_fluid);
        while (true) {
            if (r.nonfinite > 0) { st = RFB_ERR_NONFINITE; break; }
            if (r.residual <= tol) break;
            if (done >= o.max_sweeps) { st = RFB_ERR_NOT_CONVERGED; break; }
            if (o.timeout_ms > 0 && std::chrono::duration<double, std::milli>(
                                        std::chrono::steady_clock::now() - t0).count() >= o.timeout_ms) {
                set_err(h, "opts.timeout_ms reached after %lld steps", (long long)done);
                st = RFB_ERR_NOT_CONVERGED;
                break;
            }
            const int64_t n = std::min(every, o.max_sweeps - done);
            CK(h, cudaEventRecord(h->ev[0], h->stream));
            for (int64_t q = 0; q < n; ++q) {
                nernst_interior_kernel<<<h->grid, h->block, 0, h->stream>>>(
                    lattice(h), h->K, C, dtc, op.dt, h->d_s[h->s_cur], h->d_s[h->s_cur ^ 1],
                    kap0, h->kchunk);
                LAUNCHED(h);
                if (n_elec > 0) {
                    nernst_elec_kernel<<<flat_grid(n_elec), 256, 0, h->stream>>>(
                        lattice(h), h->K, C, h->d_elec, n_elec, h->d_s[h->s_cur],
                        h->d_s[h->s_cur ^ 1], h->d_eta, kap0, Vt, omega);
                    LAUNCHED(h);
                }
                h->s_cur ^= 1;
            }
            CK(h, cudaEventRecord(h->ev[1], h->stream));
            check(h, op, false);
            CK(h, cudaEventRecord(h->ev[2], h->stream));
            CK(h, cudaEventSynchronize(h->ev[2]));
            float ms_s = 0.f, ms_c = 0.f;
            CK(h, cudaEventElapsedTime(&ms_s, h->ev[0], h->ev[1]));
            CK(h, cudaEventElapsedTime(&ms_c, h->ev[1], h->ev[2]));
            sweep_ms += ms_s;
            check_ms += ms_c;
            done += n;
            ++r.checks;
            fill_result(h, op, &r, h->n_fluid);
        }
        r.sweeps = done;
        r.sweep_ms = sweep_ms;
        r.check_ms = check_ms;
        r.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                        .count();
        h->op = op;
        h->s_converged = (st == RFB_OK);
        if (res) *res = r;
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

namespace {

// N-double fields of the Butler-Volmer state in h->d_bv: 0-1 O, 2-3 R, 4-5 H
// (ping-pong), 6 phi, 7 phi before the last potential solve, 8 right-hand side of the
// potential equation, 9 kappa_c, 10 membrane kappa, 11-14 CG r, z, p, q; then 1/diag.
constexpr int BV_FIELDS = 15;
double* bv_field(rfb_soc_handle* h, int q) { return h->d_bv + (size_t)q * h->N; }

}  // namespace

rfb_status rfb_soc_solve_bv(rfb_soc_handle* h, double s_in, double eta, double tol,
                            const rfb_bv_params* bvp, const rfb_solve_opts* opts,
                            rfb_bv_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    rfb_solve_opts o;
    if (!read_opts(h, opts, &o)) return RFB_ERR_INVALID_ARG;
    if (!(s_in >= 0 && s_in <= 1)) { set_err(h, "s_in must be in [0, 1]"); return RFB_ERR_INVALID_ARG; }
    if (!std::isfinite(eta)) { set_err(h, "eta must be finite"); return RFB_ERR_INVALID_ARG; }
    if (!(tol > 0)) { set_err(h, "tol must be > 0"); return RFB_ERR_INVALID_ARG; }
    if (o.precision != RFB_PREC_FP64 || o.dt_mode != RFB_DT_LOCAL || h->kin.mode != RFB_KIN_AFFINE) {
        set_err(h, "the Butler-Volmer model needs RFB_PREC_FP64, local steps and kinetics mode 0");
        return RFB_ERR_INVALID_ARG;
    }
    rfb_bv_params P{};
    if (bvp) P = *bvp;
    if (P.D_H == 0) P.D_H = 9.3e-9;
    if (P.D_X == 0) P.D_X = 1.38e-9;
    if (P.c_H_in == 0) P.c_H_in = 50.0 * h->kin.c0;
    if (P.cg_rtol == 0) P.cg_rtol = 1e-13;
    if (P.cycle == 0) P.cycle = 100;
    if (P.max_cg == 0) P.max_cg = 100000;
    const double cX_in = P.c_H_in - 2.0 * h->kin.c0;
    if (!(P.D_H > 0) || !(P.D_X > 0) || !std::isfinite(P.D_H + P.D_X) || !(cX_in > 0) ||
        !std::isfinite(P.c_H_in) || !(P.cg_rtol > 0 && P.cg_rtol < 1) || P.cycle < 1 ||
        P.max_cg < 1 || P.start < 0 || P.start > 2 || P.reserved != 0) {
        set_err(h, "bad rfb_bv_params (diffusivities > 0, c_H_in > 2 c0, 0 < cg_rtol < 1, "
                "cycle, max_cg >= 1, start 0..2, reserved 0)");
        return RFB_ERR_INVALID_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    try {
        OpPoint op = make_op(o, s_in, eta, false);
        // model refinement needs the converged SBV state of this operating point
        const bool sbv_ok = h->have_state && h->s_converged && h->op.valid &&
                            h->op.s_in == s_in && h->op.eta == eta && h->op.beta == op.beta &&
                            h->op.inlet_bc == op.inlet_bc;
        if (P.start == 1 && !sbv_ok) {
            set_err(h, "no converged SBV state at this operating point to refine");
            return RFB_ERR_STATE;
        }
        const bool from_sbv = sbv_ok && P.start != 2;
        prepare(h, op);   // velocities * beta / h; op.A, op.B
        const int64_t N = h->N;
        if (!h->d_bv) {
            dalloc(h, &h->d_bv, (size_t)BV_FIELDS * N + N);   // + 1/diag of the CG
            dalloc(h, &h->d_bvpart, (size_t)BV_NB * NRED + 16);
        }
        double* dinv = h->d_bv + (size_t)BV_FIELDS * N;
        double* part = h->d_bvpart;
        double* sc = h->d_bvpart + (size_t)BV_NB * NRED;   // CG scalars (3) + spare
        const double VT = R_GAS * h->kin.T / FARADAY;
        const double hh = h->h * h->h;
        const double c0 = h->kin.c0;
        BVArgs A{};
        A.nx = h->nx; A.ny = h->ny; A.nz = h->nz; A.nxny = h->nxny; A.N = N;
        A.flags = h->d_flags;
        A.u = h->d_us; A.v = h->d_vs; A.w = h->d_ws; A.m = h->d_m;
        const double gin = op.inlet_bc == RFB_INLET_GHOST ? 1.0 : 2.0;
        const double Dsp[3] = {h->D, h->D, P.D_H};
        const double zsp[3] = {-2.0, -2.0, 1.0};
        const double cin[3] = {(1.0 - s_in) * c0, s_in * c0, P.c_H_in};
        const double nst[3] = {-1.0, 1.0, -2.0};
        for (int q = 0; q < 3; ++q) {
            A.sp[q].Dh = Dsp[q] / hh;
            A.sp[q].gDh = gin * Dsp[q] / hh;
            A.sp[q].g = zsp[q] * Dsp[q] * FARADAY / (R_GAS * h->kin.T * hh);
            A.sp[q].c_in = cin[q];
            A.sp[q].nst = nst[q];
            A.sp[q].zD = zsp[q] * Dsp[q];
            A.sp[q].membrane = q == 2;
        }
        A.x_zD = -P.D_X;
        A.x_cin = cX_in;
        A.lap_in = gin;
        A.kap0 = h->kin.k0 / h->h;
        A.alpha = h->kin.alpha;
        A.Vt = h->kin.n_e * (-eta) / VT;
        A.ne_VT = h->kin.n_e / VT;
        A.F = FARADAY;
        A.pre = FARADAY * FARADAY / (R_GAS * h->kin.T);
        A.D4 = 4.0 * h->D;
        A.D_H = P.D_H;
        A.D_X = P.D_X;
        A.ne_F = h->kin.n_e * FARADAY;
        A.h2 = hh;
        A.cfl = op.cfl;
        h->bv_cur = 0;
        bv_init_kernel<<<flat_grid(N), BV_TPB, 0, h->stream>>>(
            A, from_sbv ? h->d_s[h->s_cur] : nullptr, s_in, c0, bv_field(h, 0),
            bv_field(h, 2), bv_field(h, 4), bv_field(h, 6));
        LAUNCHED(h);
        h->have_bv = true;
        // tau = V_f / Q as in the SBV residual
        const double Q = op.beta * h->sum_w_in * hh;
        const double tau = Q > 0 ? (double)h->n_fluid * hh * h->h / Q
                                 : std::pow(h->nz * h->h, 2) / h->D;
        const double scale[3] = {c0, c0, P.c_H_in};
        std::vector<double> hp((size_t)BV_NB * BV_STATS);
        double hred[NRED];
        rfb_bv_result r{};
        rfb_status st = RFB_OK;
        auto check = [&]() {   // species residuals and outputs at (C, phi)
            const int cur = h->bv_cur;
            bv_check_kernel<<<BV_NB, BV_TPB, 0, h->stream>>>(
                A, bv_field(h, 0 + cur), bv_field(h, 2 + cur), bv_field(h, 4 + cur),
                bv_field(h, 6), bv_field(h, 8), bv_field(h, 9), bv_field(h, 10), part);
            LAUNCHED(h);
            finalize_kernel<<<1, 256, 0, h->stream>>>(part, BV_NB, h->d_red, 0);
            LAUNCHED(h);
            CK(h, cudaMemcpyAsync(hred, h->d_red, sizeof hred, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            double resid = 0.0;
            for (int q = 0; q < 3; ++q)
                resid = std::max(resid, tau * std::sqrt(hred[q] / (double)h->n_fluid) / scale[q]);
            r.residual = std::isfinite(hred[0] + hred[1] + hred[2]) ? resid : NAN;
            r.I_tot = h->kin.n_e * FARADAY * hh * h->h * hred[3];
            const double denom = h->kin.n_e * FARADAY * c0 * Q * (1.0 - s_in);
            r.U = denom != 0 ? r.I_tot / denom : NAN;
            r.s_out = hred[5] != 0 ? hred[4] / hred[5] : NAN;
            r.I_membrane = hred[6] * h->h;
            return hred[7];   // max |right-hand side of the potential equation|
        };
        // conjugate gradients on -K phi = -bphi, warm-started from the current phi;
        // returns the largest change of phi
        bool cg_ok = false;
        auto potential = [&](double bmax) -> double {
            double* phi = bv_field(h, 6);
            CK(h, cudaMemcpyAsync(bv_field(h, 7), phi, N * 8, cudaMemcpyDeviceToDevice, h->stream));
            double* rr = bv_field(h, 11);
            double* zz = bv_field(h, 12);
            double* pp = bv_field(h, 13);
            double* qq = bv_field(h, 14);
            bv_cg_start_kernel<<<BV_NB, BV_TPB, 0, h->stream>>>(A, bv_field(h, 9), bv_field(h, 10),
                                                                 bv_field(h, 8), phi, rr, zz, pp,
                                                                 dinv, part);
            LAUNCHED(h);
            bv_sum_kernel<<<1, BV_TPB, 0, h->stream>>>(part, BV_NB, sc + 0);
            LAUNCHED(h);
            int it = 0;
            double stats[BV_STATS] = {0, 0, 0, 0, 0, 0};
            auto read_stats = [&]() {
                bv_potential_stats_kernel<<<BV_NB, BV_TPB, 0, h->stream>>>(
                    A, bv_field(h, 9), bv_field(h, 10), bv_field(h, 8), phi, bv_field(h, 7), part);
                LAUNCHED(h);
                CK(h, cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost,
                                      h->stream));
                CK(h, cudaStreamSynchronize(h->stream));
                stats[0] = stats[1] = stats[2] = stats[5] = 0.0;
                stats[3] = INFINITY; stats[4] = -INFINITY;
                for (int b = 0; b < BV_NB; ++b) {
                    const double* q = &hp[(size_t)b * BV_STATS];
                    stats[0] = std::max(stats[0], q[0]);
                    stats[1] = std::max(stats[1], q[1]);
                    stats[2] += q[2];
                    stats[3] = std::min(stats[3], q[3]);
                    stats[4] = std::max(stats[4], q[4]);
                    stats[5] = std::max(stats[5], q[5]);
                }
            };
            // done at cg_rtol of the right-hand side, or at the rounding floor of the
            // residual (64 eps of the largest diag |phi| term), or when 20 checks in a row
            // brought no halving (stagnation at that floor)
            auto done_cg = [&]() {
                return stats[0] <= std::max(P.cg_rtol * bmax, 64.0 * 2.2e-16 * stats[5]);
            };
            read_stats();
            double best = stats[0];
            int stall = 0;
            while (!done_cg() && it < P.max_cg && stall < 20) {
                for (int k = 0; k < 50 && it < P.max_cg; ++k, ++it) {
                    bv_cg_matvec_kernel<<<BV_NB, BV_TPB, 0, h->stream>>>(
                        A, bv_field(h, 9), bv_field(h, 10), pp, qq, part);
                    bv_sum_kernel<<<1, BV_TPB, 0, h->stream>>>(part, BV_NB, sc + 1);
                    bv_cg_update_kernel<<<BV_NB, BV_TPB, 0, h->stream>>>(N, sc, phi, rr, zz, pp,
                                                                          qq, dinv, part);
                    bv_sum_kernel<<<1, BV_TPB, 0, h->stream>>>(part, BV_NB, sc + 2);
                    bv_cg_direction_kernel<<<BV_NB, BV_TPB, 0, h->stream>>>(N, sc, pp, zz);
                    bv_copy_scalar_kernel<<<1, 1, 0, h->stream>>>(sc);
                    h->launches += 6;
                }
                read_stats();
                if (!std::isfinite(stats[0])) break;
                if (stats[0] < 0.5 * best) { best = stats[0]; stall = 0; }
                else ++stall;
            }
            r.cg_iterations += it;
            r.phi_mean = stats[2] / (double)h->n_fluid;
            r.phi_min = stats[3];
            r.phi_max = stats[4];
            // the solve reached its tolerance or stalled at its rounding floor; a solve
            // cut off by max_cg does not count as converged
            cg_ok = done_cg() || stall >= 20;
            if (!cg_ok && std::isfinite(stats[0]))
                set_err(h, "potential solve: max residual %.3e after %d iterations", stats[0], it);
            return stats[1];
        };
        // From a cold start the species first relax at phi = 0 (the SBV problem) until
        // their residual is below 1e-3 (or tol): a potential solved from the far-from-
        // steady reaction currents of s = s_in would feed back exponentially through the
        // source. From the SBV state the potential is solved at once.
        bool potential_on = from_sbv;
        int64_t done = 0;
        while (true) {
            const double bmax = check();
            if (!potential_on && r.residual <= std::max(1e-3, tol)) potential_on = true;
            if (potential_on) {
                r.dphi = potential(bmax);
                ++r.cycles;
                check();
            } else {
                r.dphi = INFINITY;
            }
            if (!std::isfinite(r.residual) || (potential_on && !std::isfinite(r.dphi))) {
                st = RFB_ERR_NONFINITE;
                break;
            }
            if (r.residual <= tol && r.dphi <= tol * VT / h->kin.n_e && cg_ok) break;
            if (done >= o.max_sweeps) { st = RFB_ERR_NOT_CONVERGED; break; }
            if (o.timeout_ms > 0 && std::chrono::duration<double, std::milli>(
                                        std::chrono::steady_clock::now() - t0).count() >= o.timeout_ms) {
                set_err(h, "opts.timeout_ms reached after %lld sweeps", (long long)done);
                st = RFB_ERR_NOT_CONVERGED;
                break;
            }
            const int64_t n = std::min<int64_t>(P.cycle, o.max_sweeps - done);
            for (int64_t q = 0; q < n; ++q) {
                const int cur = h->bv_cur;
                bv_sweep_kernel<<<flat_grid(N), BV_TPB, 0, h->stream>>>(
                    A, bv_field(h, 0 + cur), bv_field(h, 2 + cur), bv_field(h, 4 + cur),
                    bv_field(h, 6), bv_field(h, 1 - cur), bv_field(h, 3 - cur),
                    bv_field(h, 5 - cur));
                LAUNCHED(h);
                h->bv_cur ^= 1;
            }
            done += n;
        }
        r.sweeps = done;
        r.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (res) *res = r;
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_get_bv_state(rfb_soc_handle* h, double* c_o, double* c_r, double* c_h,
                                double* phi, rfb_mem_kind kind) {
    rfb_status g = guard(h);
    if (g) return g;
    if (kind != RFB_MEM_HOST && kind != RFB_MEM_DEVICE) { set_err(h, "bad kind"); return RFB_ERR_INVALID_ARG; }
    if (!h->have_bv) { set_err(h, "no Butler-Volmer state: call rfb_soc_solve_bv first"); return RFB_ERR_STATE; }
    try {
        double* outs[4] = {c_o, c_r, c_h, phi};
        const int fld[4] = {0 + h->bv_cur, 2 + h->bv_cur, 4 + h->bv_cur, 6};
        for (int q = 0; q < 4; ++q) {
            if (!outs[q]) continue;
            CK(h, cudaMemcpyAsync(outs[q], bv_field(h, fld[q]), h->N * 8,
                                  kind == RFB_MEM_HOST ? cudaMemcpyDeviceToHost
                                                       : cudaMemcpyDeviceToDevice,
                                  h->stream));
        }
        CK(h, cudaStreamSynchronize(h->stream));
    } catch (Fail f) {
        return f.st;
    }
    return RFB_OK;
}

rfb_status rfb_soc_get_overpotential(rfb_soc_handle* h, double* eta_t, rfb_mem_kind kind) {
    rfb_status g = guard(h);
    if (g) return g;
    if (!eta_t || (kind != RFB_MEM_HOST && kind != RFB_MEM_DEVICE)) {
        set_err(h, "eta_t must be non-NULL and kind HOST or DEVICE");
        return RFB_ERR_INVALID_ARG;
    }
    if (!h->have_eta) {
        set_err(h, "no Nernst-model solve on the current state");
        return RFB_ERR_STATE;
    }
    try {
        CK(h, cudaMemcpyAsync(eta_t, h->d_eta, h->N * sizeof(double),
                              kind == RFB_MEM_HOST ? cudaMemcpyDeviceToHost
                                                   : cudaMemcpyDeviceToDevice,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return RFB_OK;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_reset_state(rfb_soc_handle* h) {
    rfb_status g = guard(h);
    if (g) return g;
    h->have_eta = false;
    h->have_state = false;
    h->s_converged = false;
    h->op.valid = false;
    return RFB_OK;
}

rfb_status rfb_soc_get_state(rfb_soc_handle* h, double* s, rfb_mem_kind kind) {
    rfb_status g = guard(h);
    if (g) return g;
    if (!s) { set_err(h, "s is NULL"); return RFB_ERR_INVALID_ARG; }
    if (!h->have_state) { set_err(h, "no state"); return RFB_ERR_STATE; }
    try {
        CK(h, cudaMemcpyAsync(s, h->d_s[h->s_cur], h->N * 8,
                              kind == RFB_MEM_HOST ? cudaMemcpyDeviceToHost
                                                   : cudaMemcpyDeviceToDevice,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    } catch (Fail f) {
        return f.st;
    }
    return RFB_OK;
}

rfb_status rfb_soc_set_state(rfb_soc_handle* h, const double* s, rfb_mem_kind kind) {
    rfb_status g = guard(h);
    if (g) return g;
    if (!s) { set_err(h, "s is NULL"); return RFB_ERR_INVALID_ARG; }
    if (kind != RFB_MEM_HOST && kind != RFB_MEM_DEVICE) { set_err(h, "bad kind"); return RFB_ERR_INVALID_ARG; }
    h->have_eta = false;
    try {
        const double* src = s;
        if (kind == RFB_MEM_HOST) {
            if (!h->d_stage) dalloc(h, &h->d_stage, h->N);
            CK(h, cudaMemcpyAsync(h->d_stage, s, h->N * 8, cudaMemcpyHostToDevice, h->stream));
            src = h->d_stage;
        }
        CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned long long), h->stream));
        set_state_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(h->d_flags, src, h->d_s[0],
                                                                 h->d_s[1], h->d_err, h->N);
        LAUNCHED(h);
        unsigned long long bad = 0;
        CK(h, cudaMemcpyAsync(&bad, h->d_err, sizeof bad, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->s_cur = 0;
        h->have_state = true;
        h->s_converged = false;
        if (bad) { set_err(h, "%llu non-finite state values (set to 0)", bad); return RFB_ERR_INVALID_ARG; }
    } catch (Fail f) {
        return f.st;
    }
    return RFB_OK;
}

rfb_status rfb_soc_upsample(const rfb_soc_handle* coarse, rfb_soc_handle* fine) {
    if (!coarse) { set_err(fine, "coarse is NULL"); return RFB_ERR_INVALID_ARG; }
    rfb_status g = guard(fine);
    if (g) return g;
    if (coarse->device != fine->device) {
        set_err(fine, "coarse and fine handles are on different devices");
        return RFB_ERR_INVALID_ARG;
    }
    if (fine->nx != 2 * coarse->nx || fine->ny != 2 * coarse->ny || fine->nz != 2 * coarse->nz) {
        set_err(fine, "fine dims (%d,%d,%d) must be twice the coarse dims (%d,%d,%d)", fine->nx,
                fine->ny, fine->nz, coarse->nx, coarse->ny, coarse->nz);
        return RFB_ERR_INVALID_ARG;
    }
    if (std::fabs(2.0 * fine->h - coarse->h) > 1e-12 * coarse->h) {
        set_err(fine, "fine dx must be half the coarse dx");
        return RFB_ERR_INVALID_ARG;
    }
    if (!coarse->have_state) {
        set_err(fine, "coarse handle has no state to prolong");
        return RFB_ERR_STATE;
    }
    try {
        // the coarse state is read on the fine handle's stream: order it after the
        // coarse handle's queued work
        CK(fine, cudaStreamSynchronize(coarse->stream));
        const double fill = coarse->op.valid ? coarse->op.s_in : 0.0;
        prolong_kernel<<<flat_grid(fine->N), 256, 0, fine->stream>>>(
            coarse->d_flags, coarse->d_s[coarse->s_cur], coarse->nx, coarse->ny, coarse->nz,
            fine->d_flags, fine->d_s[0], fine->d_s[1], fill);
        LAUNCHED(fine);
        CK(fine, cudaStreamSynchronize(fine->stream));
        fine->s_cur = 0;
        fine->have_state = true;
        fine->s_converged = false;
    } catch (Fail f) {
        return f.st;
    }
    return RFB_OK;
}

rfb_status rfb_soc_set_area_mult(rfb_soc_handle* h, const double* m, rfb_mem_kind kind) {
    rfb_status g = guard(h);
    if (g) return g;
    if (kind != RFB_MEM_HOST && kind != RFB_MEM_DEVICE) { set_err(h, "bad kind"); return RFB_ERR_INVALID_ARG; }
    try {
        // validate on the device (count of entries that are not finite and > 0) before
        // anything is replaced; NULL restores 1 everywhere
        const double* src = m;
        if (!m || kind == RFB_MEM_HOST) {
            if (!h->d_stage) dalloc(h, &h->d_stage, h->N);
            if (m) {
                CK(h, cudaMemcpyAsync(h->d_stage, m, h->N * 8, cudaMemcpyHostToDevice,
                                      h->stream));
            } else {
                fill_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(h->d_stage, 1.0, h->N);
                LAUNCHED(h);
            }
            src = h->d_stage;
        }
        const int sblocks = (int)std::min<int64_t>(h->nblocks, 2048);
        stats_kernel<<<sblocks, 256, 0, h->stream>>>(h->d_flags, h->d_w, src, h->N, h->nxny,
                                                     h->d_partials);
        LAUNCHED(h);
        finalize_kernel<<<1, 256, 0, h->stream>>>(h->d_partials, sblocks, h->d_red, 0);
        LAUNCHED(h);
        CK(h, cudaMemcpyAsync(h->h_red, h->d_red, NRED * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (h->h_red[4] > 0) {
            set_err(h, "area_mult must be finite and > 0 (%.0f cells are not)", h->h_red[4]);
            return RFB_ERR_INVALID_ARG;
        }
        if (!h->d_m) {   // allocated only once the values are known to be valid
            dalloc(h, &h->d_m, h->N);
            dalloc(h, &h->d_m32, h->N);
        }
        scale_kernel<<<flat_grid(h->N), 256, 0, h->stream>>>(src, h->d_m, h->d_m32, 1.0, h->N);
        LAUNCHED(h);
        CK(h, cudaStreamSynchronize(h->stream));
        h->s_converged = false;   // the operator changed; the state stays as a warm start
        ++h->area_version;
    } catch (Fail f) {
        return f.st;
    }
    return RFB_OK;
}

rfb_status rfb_soc_adjoint(rfb_soc_handle* h, rfb_objective obj, double tol,
                           const rfb_solve_opts* opts, double* d_area_mult,
                           double* d_velocity_scale, rfb_mem_kind kind,
                           rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    if (obj != RFB_OBJ_I_TOT && obj != RFB_OBJ_U && obj != RFB_OBJ_U_MT) {
        set_err(h, "unknown objective");
        return RFB_ERR_INVALID_ARG;
    }
    if (!(tol > 0)) { set_err(h, "tol must be > 0"); return RFB_ERR_INVALID_ARG; }
    if (kind != RFB_MEM_HOST && kind != RFB_MEM_DEVICE) { set_err(h, "bad kind"); return RFB_ERR_INVALID_ARG; }
    const bool umt = obj == RFB_OBJ_U_MT;
    if (umt ? !(h->have_umt_state && h->t_converged) : !(h->have_state && h->s_converged)) {
        set_err(h, umt ? "adjoint of U_mt needs a converged rfb_soc_umt first"
                       : "adjoint needs a converged rfb_soc_solve at the current operating point");
        return RFB_ERR_STATE;
    }
    rfb_solve_opts o;
    if (!read_opts(h, opts, &o)) return RFB_ERR_INVALID_ARG;
    OpPoint op = umt ? h->umt_op : h->op;
    if (!(op.beta > 0)) { set_err(h, "the adjoint needs velocity_scale > 0"); return RFB_ERR_INVALID_ARG; }
    const bool mixed = o.precision == RFB_PREC_MIXED;
    if (mixed && ((!umt && h->kin.mode != RFB_KIN_AFFINE) || h->nx % 4 != 0)) {
        set_err(h, "a mixed-precision adjoint needs kinetics mode 0 (or U_MT) and nx %% 4 == 0");
        return RFB_ERR_INVALID_ARG;
    }
    op.dt_mode = o.dt_mode;
    op.cfl = o.cfl;
    auto t0 = std::chrono::steady_clock::now();
    try {
        const int64_t N = h->N;
        if (!h->d_lam[0]) {
            dalloc(h, &h->d_lam[0], N);
            dalloc(h, &h->d_lam[1], N);
            dalloc(h, &h->d_g, N);
            dalloc(h, &h->d_grad, N);
        }
        prepare(h, op);   // dt / local dt: L and L^T share their diagonal
        const double* s = umt ? h->d_t[h->t_cur] : h->d_s[h->s_cur];
        // objective value (for the explicit beta term of U) and the scales
        rfb_solve_result fwd{};
        check(h, op, umt);
        fill_result(h, op, &fwd, umt ? h->n_fluid - h->n_elec : h->n_fluid);
        const double h3 = h->h * h->h * h->h;
        const double scale = h->kin.n_e * FARADAY * h->kin.c0 * h3;
        const double Q = op.beta * h->sum_w_in * h->h * h->h;
        double jscale = 1.0;
        if (obj == RFB_OBJ_I_TOT) jscale = scale;
        if (obj == RFB_OBJ_U) {
            const double denom = h->kin.n_e * FARADAY * h->kin.c0 * Q * (1.0 - op.s_in);
            if (!(denom != 0)) { set_err(h, "U undefined (Q = 0 or s_in = 1)"); return RFB_ERR_INVALID_ARG; }
            jscale = scale / denom;
        }
        // outlet flux sum (beta-scaled velocities / h) for U_mt's dJ/ds
        const double w_out_sum = op.beta / h->h * h->sum_w_out;
        Coef<double> C = make_coef<double>(h, op, false, op.dt_mode == RFB_DT_LOCAL);
        // dR~/ds per fiber face: -k0 B / h (affine law) or k0 K1 / h times g'(s) (mode 1)
        const double kR = C.nl ? h->kin.k0 / h->h * op.K1 : -(h->kin.k0 / h->h * op.B);
        ensure_L64(h, op);   // L^T is gathered from the assembled rows
        if (C.nl) {
            // mode 1: the Jacobian at the steady state (transport + source derivative);
            // the operator is re-assembled by the next call that needs it
            linearise64_kernel<<<flat_grid(N), 256, 0, h->stream>>>(lattice(h), C, h->K, s);
            LAUNCHED(h);
            h->L64_valid = false;
        }
        adjoint_source_kernel<<<flat_grid(N), 256, 0, h->stream>>>(lattice(h), C, umt ? 2 : 0,
                                                                   w_out_sum, kR, s, h->d_g);
        LAUNCHED(h);
        CK(h, cudaMemsetAsync(h->d_lam[0], 0, N * 8, h->stream));
        CK(h, cudaMemsetAsync(h->d_lam[1], 0, N * 8, h->stream));
        int cur = 0;
        const int64_t every = o.check_every > 0 ? o.check_every : (mixed ? 200 : 100);
        rfb_solve_result r{};
        rfb_status st = RFB_OK;
        double rel = INFINITY;
        int64_t done = 0;
        // FP64 adjoint residual of d_lam[cur] (relative to ||g||)
        auto check64 = [&]() {
            adjoint64c_kernel<1><<<h->grid, h->block, 0, h->stream>>>(
                lattice(h), h->K, C.dtc, op.dt, h->d_lam[cur], nullptr, h->d_g, h->d_partials,
                op.umt, h->kchunk);
            LAUNCHED(h);
            reduce_readback(h, 0);
            ++r.checks;
            rel = h->h_red[1] > 0 ? std::sqrt(h->h_red[0] / h->h_red[1]) : 0.0;
        };
        auto time_up = [&]() {
            return o.timeout_ms > 0 &&
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                           .count() >= o.timeout_ms;
        };
        if (mixed) {
            // FP32 transposed correction sweeps on delta, double-float defects
            // r = g + L^T lam, FP64 confirmation of the cycle that meets tol
            ensure_L2F(h, op);
            if (!h->d_gdf) dalloc(h, &h->d_gdf, N);
            if (!h->d_sdf[0]) {
                dalloc(h, &h->d_sdf[0], N);
                dalloc(h, &h->d_sdf[1], N);
            }
            split64_kernel<<<flat_grid(N), 256, 0, h->stream>>>(h->d_g, h->d_gdf, N);
            LAUNCHED(h);
            CK(h, cudaMemsetAsync(h->d_sdf[0], 0, N * sizeof(float2), h->stream));
            h->df_cur = 0;
            L2F K2;
            for (int q = 0; q < 6; ++q) K2.f[q] = h->d_L2F + q * (size_t)N;
            K2.diag = h->d_L2F + 6 * (size_t)N;
            K2.b = h->d_L2F + 7 * (size_t)N;
            const Coef<float> C32 = make_coef<float>(h, op, true, false);
            auto df_check = [&](bool fuse) {
                const int dc = h->df_cur;
                if (fuse) {
                    check_df_adjoint_kernel<true><<<h->grid, h->block, 0, h->stream>>>(
                        lattice(h), K2, h->d_sdf[dc], h->d_delta[0], h->d_sdf[dc ^ 1], h->d_gdf,
                        h->d_r32, h->d_partials, op.umt, h->kchunk);
                    h->df_cur ^= 1;
                } else {
                    check_df_adjoint_kernel<false><<<h->grid, h->block, 0, h->stream>>>(
                        lattice(h), K2, h->d_sdf[dc], nullptr, nullptr, h->d_gdf, h->d_r32,
                        h->d_partials, op.umt, h->kchunk);
                }
                LAUNCHED(h);
                reduce_readback(h, 0);
                ++r.checks;
                rel = h->h_red[1] > 0 ? std::sqrt(h->h_red[0] / h->h_red[1]) : 0.0;
            };
            auto join_and_check = [&]() {
                join64_kernel<<<flat_grid(N), 256, 0, h->stream>>>(h->d_sdf[h->df_cur],
                                                                   h->d_lam[cur], N);
                LAUNCHED(h);
                check64();
            };
            CK(h, cudaMemsetAsync(tb_err_word(h), 0, sizeof(unsigned int), h->stream));
            df_check(false);
            bool joined = false;
            while (true) {
                if (h->h_red[6] > 0) { st = RFB_ERR_NONFINITE; break; }
                if (rel <= tol) {
                    if (joined) break;
                    join_and_check();
                    joined = true;
                    continue;
                }
                if (done >= o.max_sweeps) { st = RFB_ERR_NOT_CONVERGED; break; }
                if (time_up()) {
                    set_err(h, "opts.timeout_ms reached after %lld adjoint sweeps", (long long)done);
                    st = RFB_ERR_NOT_CONVERGED;
                    break;
                }
                const int64_t n = std::min(every, o.max_sweeps - done);
                sweeps32_adjoint(h, op, C32, n);
                df_check(true);
                joined = false;
                done += n;
            }
            if (!joined) {
                const bool bad = st == RFB_ERR_NONFINITE;
                join_and_check();
                if (!bad && h->h_red[6] > 0) st = RFB_ERR_NONFINITE;
            }
            unsigned int tb_bad = 0;
            CK(h, cudaMemcpyAsync(&tb_bad, tb_err_word(h), sizeof tb_bad, cudaMemcpyDeviceToHost,
                                  h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            if (tb_bad) {
                set_err(h, "a TMA stage of the two-sweep kernel did not arrive in time");
                st = RFB_ERR_CUDA;
            }
        }
        while (!mixed) {
            adjoint64c_kernel<1><<<h->grid, h->block, 0, h->stream>>>(
                lattice(h), h->K, C.dtc, op.dt, h->d_lam[cur], nullptr, h->d_g, h->d_partials,
                op.umt, h->kchunk);
            LAUNCHED(h);
            reduce_readback(h, 0);
            ++r.checks;
            rel = h->h_red[1] > 0 ? std::sqrt(h->h_red[0] / h->h_red[1]) : 0.0;
            if (h->h_red[6] > 0) { st = RFB_ERR_NONFINITE; break; }
            if (rel <= tol) break;
            if (done >= o.max_sweeps) { st = RFB_ERR_NOT_CONVERGED; break; }
            if (o.timeout_ms > 0 &&
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                        .count() >= o.timeout_ms) {
                set_err(h, "opts.timeout_ms reached after %lld adjoint sweeps", (long long)done);
                st = RFB_ERR_NOT_CONVERGED;
                break;
            }
            const int64_t n = std::min(every, o.max_sweeps - done);
            for (int64_t q = 0; q < n; ++q) {
                adjoint64c_kernel<0><<<h->grid, h->block, 0, h->stream>>>(
                    lattice(h), h->K, C.dtc, op.dt, h->d_lam[cur], h->d_lam[cur ^ 1], h->d_g,
                    nullptr, op.umt, h->kchunk);
                LAUNCHED(h);
                cur ^= 1;
            }
            done += n;
        }
        // gradients
        const double kap0A = umt ? 0.0 : h->kin.k0 / h->h * (C.nl ? op.K1 : op.A);
        const double kap0B = umt ? 0.0 : h->kin.k0 / h->h * op.B;
        gradient_kernel<<<h->grid, h->block, 0, h->stream>>>(
            lattice(h), C, s, h->d_lam[cur], kap0A, kap0B, jscale, 1.0,
            umt ? nullptr : h->d_grad, h->d_partials, h->kchunk);
        LAUNCHED(h);
        reduce_readback(h, 0);
        double dbeta = jscale * h->h_red[0] / op.beta;
        if (obj == RFB_OBJ_U) dbeta -= fwd.U / op.beta;
        if (umt) CK(h, cudaMemsetAsync(h->d_grad, 0, N * 8, h->stream));
        if (d_area_mult) {
            CK(h, cudaMemcpyAsync(d_area_mult, h->d_grad, N * 8,
                                  kind == RFB_MEM_HOST ? cudaMemcpyDeviceToHost
                                                       : cudaMemcpyDeviceToDevice,
                                  h->stream));
        }
        CK(h, cudaStreamSynchronize(h->stream));
        if (d_velocity_scale) *d_velocity_scale = dbeta;
        r.sweeps = done;
        r.residual = rel;
        r.I_tot = fwd.I_tot;
        r.U = fwd.U;
        r.outlet_mean = fwd.outlet_mean;
        r.dt = op.dt;
        r.tau = fwd.tau;
        r.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (res) *res = r;
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

rfb_status rfb_soc_info(const rfb_soc_handle* h, int64_t* n_cells, int64_t* n_fluid) {
    if (!h) return RFB_ERR_INVALID_ARG;
    if (n_cells) *n_cells = h->N;
    if (n_fluid) *n_fluid = h->n_fluid;
    return RFB_OK;
}

int64_t rfb_soc_kernel_launches(const rfb_soc_handle* h) { return h ? h->launches : 0; }

rfb_status rfb_selftest_bounded_wait(int64_t spin_limit, int32_t* gave_up) {
    if (!gave_up || spin_limit < 1 || spin_limit > ((int64_t)1 << 26)) {
        g_create_error = "spin_limit must be in [1, 2^26] and gave_up non-NULL";
        return RFB_ERR_INVALID_ARG;
    }
    (void)cudaGetLastError();
    unsigned int* d = nullptr;
    unsigned int hv[2] = {0, 0};
    cudaError_t e = cudaMalloc((void**)&d, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) {
        mbar_timeout_probe_kernel<<<1, 64>>>((unsigned long long)spin_limit, d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hv, d, sizeof hv, cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        g_create_error = std::string("bounded-wait self-test: ") + cudaGetErrorString(e);
        return RFB_ERR_CUDA;
    }
    *gave_up = (hv[0] == 1u && hv[1] == 1u) ? 1 : 0;
    return RFB_OK;
}

rfb_status rfb_soc_tuned_fp32_kernel(const rfb_soc_handle* h, int32_t* kernel,
                                     double* plain_ms_per_sweep,
                                     double* blocked_ms_per_sweep) {
    if (!h) return RFB_ERR_INVALID_ARG;
    int32_t k = 0;
    if (h->tb_mode == 0) k = 1;
    else if (h->tb_mode == 1 || h->tb_variant >= 0) {
        const int v = std::max(h->tb_variant, 0);
        k = (v & 4 ? (v & 2 ? 9 : 7) : (v & 2 ? 5 : 3)) + (v & 1);
    }
    if (kernel) *kernel = k;
    if (plain_ms_per_sweep) *plain_ms_per_sweep = h->tb_tuned_plain_ms;
    if (blocked_ms_per_sweep) *blocked_ms_per_sweep = h->tb_tuned_tb_ms;
    return RFB_OK;
}

}  // extern "C"

// =====================================================================================
// Allocation-free evaluation of the outputs
//
// rfb_soc_current needs scratch for its per-block partial sums; it uses a buffer that
// rfb_soc_create allocated. Some callers cannot allocate device memory at the moment
// they want the outputs: a runtime whose caching allocator already owns the device's
// memory budget, or a monitor on a latency-critical path that must not pay for the
// implicit device synchronisation of cudaMalloc/cudaFree. rfb_soc_current_noalloc serves
// them: the matrix-free FP64 check kernel (check_kernel, which builds each cell's
// coefficients from the face velocities; rfb_soc_current runs check64c_kernel on the
// assembled operator, so the two agree up to rounding) and the same fixed-order
// reduction, but the scratch is the file-scope array below, present on every device that
// loads this library until the process exits.
// =====================================================================================
namespace {

// 8192 blocks x 8 partial sums, then the 8 final sums: 8200 doubles = 65,600 bytes.
constexpr int64_t NOALLOC_MAX_BLOCKS = 8192;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS * NRED + NRED];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[256] = {};   // device address of g_noalloc_scratch, per device

// Device address of the scratch on h's device, looked up with that device current (h's
// device is made current by guard()). In host code the symbol's name is only a host-side
// stand-in, so kernels must be given this address. It is looked up again on every call
// made outside a stream capture (a cudaDeviceReset reloads the module, and the array may
// then sit elsewhere); during a capture the address from the last uncaptured call on
// that device is used, so the first call on a device must come before any capture.
rfb_status noalloc_scratch(rfb_soc_handle* h, double** out) {
    if (h->device < 0 || h->device >= 256) {
        set_err(h, "device ordinal %d out of range", h->device);
        return RFB_ERR_CUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(h->stream, &cap);
    if (ce != cudaSuccess) {
        set_err(h, "cudaStreamIsCapturing failed: %s", cudaGetErrorString(ce));
        return RFB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap != cudaStreamCaptureStatusNone && !g_noalloc_addr[h->device]) {
        set_err(h, "the first rfb_soc_current_noalloc call on a device must come before any "
                "stream capture");
        return RFB_ERR_STATE;
    }
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_err(h, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s",
                    cudaGetErrorString(e));
            return RFB_ERR_CUDA;
        }
        g_noalloc_addr[h->device] = (double*)p;
    }
    *out = g_noalloc_addr[h->device];
    return RFB_OK;
}

}  // namespace

extern "C" rfb_status rfb_soc_current_noalloc(rfb_soc_handle* h, rfb_solve_result* res) {
    rfb_status g = guard(h);
    if (g) return g;
    if (!res) { set_err(h, "res is NULL"); return RFB_ERR_INVALID_ARG; }
    if (!h->have_state || !h->op.valid) {
        set_err(h, "no state / operating point: call rfb_soc_solve or rfb_soc_step first");
        return RFB_ERR_STATE;
    }
    if (h->nblocks > NOALLOC_MAX_BLOCKS) {
        set_err(h, "lattice needs %lld reduction blocks; the static scratch of "
                "rfb_soc_current_noalloc holds %lld (use rfb_soc_current)",
                (long long)h->nblocks, (long long)NOALLOC_MAX_BLOCKS);
        return RFB_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    rfb_status st = noalloc_scratch(h, &scratch);
    if (st) return st;
    try {
        // Every partial slot read by finalize_kernel is written by check_kernel in this
        // call, and finalize_kernel writes every final slot, so nothing left over from an
        // earlier call is read and nothing has to be cleared first.
        const OpPoint op = h->op;
        rescale_velocities(h, op.beta);   // allocates nothing
        Coef<double> C = make_coef<double>(h, op, false, false);
        double* partials = scratch;
        double* sums = scratch + NOALLOC_MAX_BLOCKS * NRED;
        check_kernel<false, false><<<h->grid, h->block, 0, h->stream>>>(
            lattice(h), C, h->d_s[h->s_cur], nullptr, nullptr, nullptr, partials, h->kchunk);
        LAUNCHED(h);
        finalize_kernel<<<1, 256, 0, h->stream>>>(partials, h->nblocks, sums, 0);
        LAUNCHED(h);
        double host_sums[NRED];
        CK(h, cudaMemcpyAsync(host_sums, sums, sizeof host_sums, cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        rfb_solve_result r{};
        r.checks = 1;
        fill_result(h, op, &r, h->n_fluid, host_sums);
        *res = r;
        return r.nonfinite ? RFB_ERR_NONFINITE : RFB_OK;
    } catch (Fail f) {
        return f.st;
    }
}

// =====================================================================================
// Batches (many lattices, one persistent launch per sweep, one CUDA graph per cycle)
// =====================================================================================
namespace {

// Cycle budget of one launch of the device-driven batch loop (set by the host before each
// launch) and the cycles run (counted on the device).
struct BatchLoop {
    int cycles;
    int max_cycles;
    int n_inst;
    int pad_;
};

// Last node of the loop body: counts the cycle and sets the while node's condition, 1 while
// a lattice is still active (not converged, finite) and the budget is not spent.
__global__ void batch_loop_kernel(const BatchCtl* __restrict__ ctl, BatchLoop* __restrict__ lp,
                                  cudaGraphConditionalHandle hc) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < lp->n_inst; q += blockDim.x)
        if (!ctl[q].converged && !ctl[q].nonfinite) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int c = lp->cycles + 1;
        lp->cycles = c;
        cudaGraphSetConditional(hc, (any && c < lp->max_cycles) ? 1u : 0u);
    }
}

}  // namespace

struct rfb_batch {
    std::vector<rfb_soc_handle*> hs;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    BatchInst* d_insts = nullptr;
    BatchCtl* d_ctl = nullptr;
    BatchCtl* h_ctl = nullptr;          // pinned
    BatchItem* d_items = nullptr;
    int* d_item_begin = nullptr;
    double* d_partials = nullptr;
    int n_items = 0;
    int items_kchunk = -1;
    std::vector<int> item_begin;
    int grid_blocks = 0;             // blocks of the sweep launch (autotuned)
    int grid_blocks_resident = 0;    // SMs x resident blocks per SM
    int tuned_grid = 0;
    // autotuner results
    int tuned_kchunk = 0;
    int tuned_every = 0;
    double tuned_sweep_ms = 0, tuned_check_ms = 0;
    cudaGraphExec_t exec = nullptr;
    int exec_every = 0;
    bool exec_df = false;
    // defects in double-float (check_df arithmetic) during the cycles, FP64 once at the end
    bool df = false;
    // device-driven loop: a graph whose while node repeats the cycle until every lattice
    // has converged or the launch's cycle budget is spent
    cudaGraphExec_t loop_exec = nullptr;
    int loop_every = 0;
    bool loop_df = false;
    BatchLoop* d_loop = nullptr;
    BatchLoop* h_loop = nullptr;         // pinned
    // two-sweep passes over every lattice (local steps, every lattice nz >= 2): per-lattice
    // tensor maps (boxes for 128- and for 64-column tiles), (lattice, tile, z chunk) items,
    // tile width, chunk length and stage count (autotuned)
    BatchTBD* d_tbd = nullptr;           // 136-column boxes
    BatchTBD* d_tbdn = nullptr;          // 72-column boxes
    BatchTBItem* d_tbitems = nullptr;
    int n_tbitems = 0;
    int tb_lc = 0;                       // chunk length of the built item list
    int tb_txi = 128;                    // interior columns of a tile (128 or 64)
    int tb_nst = 0;                      // 0: one-sweep kernel; 3 / 4: passes, stages
    int sms = 152;
    int tuned_mode = -1;                 // kernel choice the tuning was made for
    unsigned int* d_tberr = nullptr;     // set if a stage of a pass never arrives
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::string err;
    int64_t launches = 0;
};

namespace {

void bset_err(rfb_batch* b, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
}

#define BCK(b, call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            bset_err((b), "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                     __FILE__, __LINE__);                                              \
            throw Fail{e_ == cudaErrorMemoryAllocation ? RFB_ERR_OOM : RFB_ERR_CUDA};  \
        }                                                                              \
    } while (0)

#define BLAUNCHED(b)                                                                    \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            bset_err((b), "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),  \
                     __FILE__, __LINE__);                                              \
            throw Fail{RFB_ERR_CUDA};                                                  \
        }                                                                              \
        ++(b)->launches;                                                               \
    } while (0)

// Work items of every lattice for a z-chunk length; item_begin[i] .. item_begin[i+1]
// are lattice i's items (contiguous, in x-fastest tile order).
void build_items(rfb_batch* b, int kchunk) {
    if (b->items_kchunk == kchunk) return;
    std::vector<BatchItem> items;
    b->item_begin.assign(1, 0);
    for (size_t q = 0; q < b->hs.size(); ++q) {
        const rfb_soc_handle* h = b->hs[q];
        // runs of 1024 consecutive cells of the flattened x-y plane (no x-tile waste on
        // lattices whose width is not a multiple of 128)
        const int groups = h->nxny / 4;
        for (int kb = 0; kb < h->nz; kb += kchunk)
            for (int g0 = 0; g0 < groups; g0 += VBX * VBY)
                items.push_back(BatchItem{(int)q, g0, 0, kb, std::min(kb + kchunk, h->nz)});
        b->item_begin.push_back((int)items.size());
    }
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_item_begin) cudaFree(b->d_item_begin);
    if (b->d_partials) cudaFree(b->d_partials);
    b->d_items = nullptr; b->d_item_begin = nullptr; b->d_partials = nullptr;
    BCK(b, cudaMalloc((void**)&b->d_items, items.size() * sizeof(BatchItem)));
    BCK(b, cudaMalloc((void**)&b->d_item_begin, b->item_begin.size() * sizeof(int)));
    BCK(b, cudaMalloc((void**)&b->d_partials, items.size() * NRED * sizeof(double)));
    BCK(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem),
                      cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(b->d_item_begin, b->item_begin.data(), b->item_begin.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    b->items_kchunk = kchunk;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->loop_exec) { cudaGraphExecDestroy(b->loop_exec); b->loop_exec = nullptr; }
}

// Items of the batched two-sweep pass for a z-chunk length and tile width: per lattice,
// chunk-major with the tiles of a chunk consecutive.
void build_tb_items(rfb_batch* b, int lc, int txi) {
    if (b->tb_lc == lc && b->tb_txi == txi) return;
    std::vector<BatchTBItem> items;
    for (size_t q = 0; q < b->hs.size(); ++q) {
        const rfb_soc_handle* h = b->hs[q];
        const int tiles = ((h->nx + txi - 1) / txi) * ((h->ny + TB_TYI - 1) / TB_TYI);
        for (int kb = 0; kb < h->nz; kb += lc)
            for (int t = 0; t < tiles; ++t)
                items.push_back(BatchTBItem{(int)q, t, kb, std::min(kb + lc, h->nz)});
    }
    if (b->d_tbitems) cudaFree(b->d_tbitems);
    b->d_tbitems = nullptr;
    BCK(b, cudaMalloc((void**)&b->d_tbitems, items.size() * sizeof(BatchTBItem)));
    BCK(b, cudaMemcpy(b->d_tbitems, items.data(), items.size() * sizeof(BatchTBItem),
                      cudaMemcpyHostToDevice));
    b->n_tbitems = (int)items.size();
    b->tb_lc = lc;
    b->tb_txi = txi;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->loop_exec) { cudaGraphExecDestroy(b->loop_exec); b->loop_exec = nullptr; }
}

void batch_sweeps(rfb_batch* b, int n, bool local) {
    if (b->tb_nst) {   // two-sweep passes (n even); pass p reads delta[p & 1]
        for (int q = 0; q < n / 2; ++q) {
            if (b->tb_txi == 64)   // two CTAs per SM
                batch_tbd_kernel<3, 64><<<2 * b->sms, TBDGeom<64>::THREADS, tbd_smem<3, 64>(),
                                          b->stream>>>(b->d_tbdn, b->d_insts, b->d_tbitems,
                                                       b->n_tbitems, q & 1, b->d_tberr);
            else if (b->tb_nst == 4)
                batch_tbd_kernel<4, 128><<<b->sms, TB_THREADS, tbd_smem<4>(), b->stream>>>(
                    b->d_tbd, b->d_insts, b->d_tbitems, b->n_tbitems, q & 1, b->d_tberr);
            else
                batch_tbd_kernel<3, 128><<<b->sms, TB_THREADS, tbd_smem<3>(), b->stream>>>(
                    b->d_tbd, b->d_insts, b->d_tbitems, b->n_tbitems, q & 1, b->d_tberr);
            BLAUNCHED(b);
        }
        return;
    }
    for (int q = 0; q < n; ++q) {
        if (local)
            batch_sweep_kernel<true><<<b->grid_blocks, dim3(VBX, VBY), 0, b->stream>>>(
                b->d_insts, b->d_items, b->n_items, q & 1);
        else
            batch_sweep_kernel<false><<<b->grid_blocks, dim3(VBX, VBY), 0, b->stream>>>(
                b->d_insts, b->d_items, b->n_items, q & 1);
        BLAUNCHED(b);
    }
}

// the check kernel of every active lattice (double-float defects when b->df, else FP64),
// item partials only
void batch_check_items(rfb_batch* b, bool fused) {
    if (b->df && fused)
        batch_check_df_kernel<true><<<b->grid_blocks, dim3(BX, BY), 0, b->stream>>>(
            b->d_insts, b->d_items, b->n_items, b->d_partials);
    else if (b->df)
        batch_check_df_kernel<false><<<b->grid_blocks, dim3(BX, BY), 0, b->stream>>>(
            b->d_insts, b->d_items, b->n_items, b->d_partials);
    else if (fused)
        batch_check_kernel<true><<<b->grid_blocks, dim3(BX, BY), 0, b->stream>>>(
            b->d_insts, b->d_items, b->n_items, b->d_partials);
    else
        batch_check_kernel<false><<<b->grid_blocks, dim3(BX, BY), 0, b->stream>>>(
            b->d_insts, b->d_items, b->n_items, b->d_partials);
    BLAUNCHED(b);
}

void batch_check(rfb_batch* b, bool fused, int sweeps_done) {
    batch_check_items(b, fused);
    batch_finalize_kernel<<<(int)b->hs.size(), 256, 0, b->stream>>>(
        b->d_insts, b->d_item_begin, b->d_partials, b->d_ctl, fused ? 1 : 0, sweeps_done);
    BLAUNCHED(b);
}

// One correction cycle: delta = 0, `every` sweeps, fused FP64 check, bookkeeping, and
// (to_host) the control block copied to the host.
void batch_cycle(rfb_batch* b, int every, bool local, bool to_host = true) {
    batch_zero_kernel<<<152 * 4, 256, 0, b->stream>>>(b->d_insts, (int)b->hs.size());
    BLAUNCHED(b);
    batch_sweeps(b, every, local);
    batch_check(b, true, every);
    if (to_host)
        BCK(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, b->hs.size() * sizeof(BatchCtl),
                               cudaMemcpyDeviceToHost, b->stream));
}

// The device-driven solve graph: one conditional while node whose body is a cycle
// followed by batch_loop_kernel, which counts the cycle and keeps the loop going while a
// lattice is still active and the launch's cycle budget (BatchLoop::max_cycles, written
// by the host before each launch) is not spent. No host round trip between cycles.
void build_loop_graph(rfb_batch* b, int every, bool local) {
    if (b->loop_exec && b->loop_every == every && b->loop_df == b->df) return;
    if (b->loop_exec) { cudaGraphExecDestroy(b->loop_exec); b->loop_exec = nullptr; }
    cudaGraph_t g = nullptr;
    BCK(b, cudaGraphCreate(&g, 0));
    try {
        cudaGraphConditionalHandle hc;
        BCK(b, cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        BCK(b, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        BCK(b, cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = b->launches;
        try {
            batch_cycle(b, every, local, false);
            batch_loop_kernel<<<1, 32, 0, b->stream>>>(b->d_ctl, b->d_loop, hc);
            BLAUNCHED(b);
        } catch (Fail) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(b->stream, &dummy);
            throw;
        }
        b->launches = l0;   // counted when run
        cudaGraph_t captured = nullptr;
        BCK(b, cudaStreamEndCapture(b->stream, &captured));
        BCK(b, cudaGraphInstantiate(&b->loop_exec, g, 0));
    } catch (Fail) {
        cudaGraphDestroy(g);
        throw;
    }
    cudaGraphDestroy(g);
    b->loop_every = every;
    b->loop_df = b->df;
}

// Project-written autotuner: for each candidate z-chunk of the work items, time a few
// persistent sweeps of the whole batch (CUDA events) and keep the fastest; then set the
// sweeps per cycle so that the FP64 check costs about 3% of a cycle.
// mode: 0 fastest of both kernels, 1 one-sweep kernel only, 2 two-sweep passes only
void autotune(rfb_batch* b, bool local, std::vector<BatchInst>& insts0, int mode) {
    // candidates: z-chunk of the items x grid size (1x / 2x the resident blocks, walking
    // the item list persistently, or one block per item)
    const int cands[] = {8, 16, 32, 64};
    const int resident = b->grid_blocks_resident;
    float best = 1e30f;
    int best_k = 16, best_grid = resident;
    for (int kc : cands) {
        build_items(b, kc);
        const int grids[] = {resident, 2 * resident, b->n_items};
        for (int gsz : grids) {
            b->grid_blocks = std::max(1, std::min(gsz, b->n_items));
            batch_sweeps(b, 2, local);   // warm-up
            BCK(b, cudaEventRecord(b->ev[0], b->stream));
            batch_sweeps(b, 4, local);
            BCK(b, cudaEventRecord(b->ev[1], b->stream));
            BCK(b, cudaEventSynchronize(b->ev[1]));
            float ms = 0;
            BCK(b, cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
            if (ms < best) { best = ms; best_k = kc; best_grid = gsz; }
        }
    }
    build_items(b, best_k);
    b->grid_blocks = std::max(1, std::min(best_grid, b->n_items));
    b->tuned_grid = best_grid;
    b->tuned_kchunk = best_k;
    b->tuned_sweep_ms = best / 4.0;
    // two-sweep passes (local steps and tensor maps in place): chunk length x (tile width,
    // stages): 128-column tiles with three or four stages (one CTA per SM), 64-column tiles
    // with three (two CTAs per SM; lattices narrower than 128 columns waste less of a tile)
    b->tb_nst = 0;
    if (mode >= 2) best = 1e30f;
    if (b->d_tbd && mode != 1) {
        float best_tb = 1e30f;
        int bl = 0, bn = 0, bw = 128;
        const int shapes[3][2] = {{128, 3}, {128, 4}, {64, 3}};
        for (int lc : {16, 32, 64}) {
            for (const auto& sh : shapes) {
                if ((mode == 3 && sh[0] != 128) || (mode == 4 && sh[0] != 64)) continue;
                build_tb_items(b, lc, sh[0]);
                b->tb_nst = sh[1];
                batch_sweeps(b, 2, local);   // warm-up
                BCK(b, cudaEventRecord(b->ev[0], b->stream));
                batch_sweeps(b, 4, local);
                BCK(b, cudaEventRecord(b->ev[1], b->stream));
                BCK(b, cudaEventSynchronize(b->ev[1]));
                float ms = 0;
                BCK(b, cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
                if (ms < best_tb) { best_tb = ms; bl = lc; bn = sh[1]; bw = sh[0]; }
            }
        }
        b->tb_nst = 0;
        if (best_tb < best || mode >= 2) {
            build_tb_items(b, bl, bw);
            b->tb_nst = bn;
            b->tuned_sweep_ms = best_tb / 4.0;
        }
    }
    BCK(b, cudaEventRecord(b->ev[0], b->stream));
    batch_check_items(b, false);
    BCK(b, cudaEventRecord(b->ev[1], b->stream));
    BCK(b, cudaEventSynchronize(b->ev[1]));
    float cms = 0;
    BCK(b, cudaEventElapsedTime(&cms, b->ev[0], b->ev[1]));
    b->tuned_check_ms = cms;
    int every = (int)std::ceil(cms / (0.03 * std::max(1e-6, b->tuned_sweep_ms)));
    every = std::max(20, std::min(400, every + (every & 1)));
    if (b->tb_nst) every = (every + 3) / 4 * 4;   // whole passes, result in delta[0]
    b->tuned_every = every;
    // the tuning sweeps touched delta only; restore the descriptors (cur / active)
    BCK(b, cudaMemcpy(b->d_insts, insts0.data(), insts0.size() * sizeof(BatchInst),
                      cudaMemcpyHostToDevice));
}

}  // namespace

extern "C" {

rfb_status rfb_soc_batch_create(rfb_soc_handle* const* hs, int n, rfb_batch** out) {
    if (!out) return RFB_ERR_INVALID_ARG;
    *out = nullptr;
    g_create_error.clear();
    if (!hs || n < 1) { g_create_error = "need at least one handle"; return RFB_ERR_INVALID_ARG; }
    for (int q = 0; q < n; ++q) {
        if (!hs[q]) { g_create_error = "NULL handle"; return RFB_ERR_INVALID_ARG; }
        if (hs[q]->device != hs[0]->device) { g_create_error = "handles on different devices"; return RFB_ERR_INVALID_ARG; }
        if (hs[q]->nx % 4 != 0) { g_create_error = "batched lattices need nx % 4 == 0"; return RFB_ERR_INVALID_ARG; }
        if (hs[q]->kin.mode != RFB_KIN_AFFINE) { g_create_error = "batched solves need kinetics mode 0 (FP32 correction sweeps)"; return RFB_ERR_INVALID_ARG; }
        for (int p = 0; p < q; ++p)
            if (hs[p] == hs[q]) { g_create_error = "a handle appears twice"; return RFB_ERR_INVALID_ARG; }
    }
    rfb_batch* b = new rfb_batch();
    b->hs.assign(hs, hs + n);
    b->device = hs[0]->device;
    try {
        BCK(b, cudaSetDevice(b->device));
        // a stream of its own: the cycle is captured into a CUDA graph, which the legacy
        // default stream does not allow
        BCK(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
        BCK(b, cudaMalloc((void**)&b->d_insts, n * sizeof(BatchInst)));
        BCK(b, cudaMalloc((void**)&b->d_ctl, n * sizeof(BatchCtl)));
        BCK(b, cudaMallocHost((void**)&b->h_ctl, n * sizeof(BatchCtl)));
        BCK(b, cudaMalloc((void**)&b->d_loop, sizeof(BatchLoop)));
        BCK(b, cudaMallocHost((void**)&b->h_loop, sizeof(BatchLoop)));
        BCK(b, cudaMalloc((void**)&b->d_tberr, sizeof(unsigned int)));
        BCK(b, cudaEventCreate(&b->ev[0]));
        BCK(b, cudaEventCreate(&b->ev[1]));
        int sms = 152, per = 4;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_sweep_kernel<true>, VBX * VBY, 0);
        b->grid_blocks = sms * std::max(1, per);
        b->grid_blocks_resident = b->grid_blocks;
    } catch (Fail f) {
        g_create_error = b->err;
        rfb_soc_batch_destroy(b);
        return f.st;
    }
    *out = b;
    return RFB_OK;
}

rfb_status rfb_soc_batch_destroy(rfb_batch* b) {
    if (!b) return RFB_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->loop_exec) cudaGraphExecDestroy(b->loop_exec);
    void* ptrs[] = {b->d_insts, b->d_ctl,  b->d_items,  b->d_item_begin, b->d_partials,
                    b->d_loop,  b->d_tbd,  b->d_tbdn, b->d_tbitems, b->d_tberr};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_loop) cudaFreeHost(b->h_loop);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->stream && b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return RFB_OK;
}

const char* rfb_soc_batch_last_error(const rfb_batch* b) {
    return b ? b->err.c_str() : g_create_error.c_str();
}

rfb_status rfb_soc_batch_solve(rfb_batch* b, const double* s_in, const double* eta,
                               const double* tol, const rfb_solve_opts* opts,
                               rfb_solve_result* res, rfb_batch_info* info) {
    if (!b) return RFB_ERR_INVALID_ARG;
    b->err.clear();
    if (!s_in || !eta || !tol) { bset_err(b, "s_in, eta and tol are required"); return RFB_ERR_INVALID_ARG; }
    const int n = (int)b->hs.size();
    rfb_solve_opts o;
    if (!read_opts(b->hs[0], opts, &o)) { b->err = b->hs[0]->err; return RFB_ERR_INVALID_ARG; }
    if (o.precision != RFB_PREC_MIXED) {
        bset_err(b, "batched solves run FP32 correction sweeps: precision must be RFB_PREC_MIXED");
        return RFB_ERR_UNSUPPORTED;
    }
    for (int q = 0; q < n; ++q) {
        if (!(s_in[q] >= 0 && s_in[q] <= 1) || !std::isfinite(eta[q]) || !(tol[q] > 0)) {
            bset_err(b, "lattice %d: need 0 <= s_in <= 1, finite eta, tol > 0", q);
            return RFB_ERR_INVALID_ARG;
        }
    }
    const bool local = o.dt_mode == RFB_DT_LOCAL;
    auto t0 = std::chrono::steady_clock::now();
    try {
        (void)cudaGetLastError();
        BCK(b, cudaSetDevice(b->device));
        std::vector<BatchInst> insts(n);
        std::vector<BatchCtl> ctl(n);
        std::vector<OpPoint> ops(n);
        for (int q = 0; q < n; ++q) {
            rfb_soc_handle* h = b->hs[q];
            OpPoint op = make_op(o, s_in[q], eta[q], false);
            try {
                prepare(h, op);
                if (!h->have_state) init_state(h, false, op.s_in);
                CK(h, cudaStreamSynchronize(h->stream));
            } catch (Fail f) {
                bset_err(b, "lattice %d: %s", q, h->err.c_str());
                throw;
            }
            h->op = op;
            h->s_converged = false;
            ops[q] = op;
            BatchInst& I = insts[q];
            std::memset(&I, 0, sizeof I);
            I.L = lattice(h);
            I.C32 = make_coef<float>(h, op, true, false);
            I.C64 = make_coef<double>(h, op, false, false);
            I.delta[0] = h->d_delta[0];
            I.delta[1] = h->d_delta[1];
            I.r32 = h->d_r32;
            I.s64[0] = h->d_s[0];
            I.s64[1] = h->d_s[1];
            I.cfl = (float)op.cfl;
            I.active = 1;
            I.cur = h->s_cur;
            BatchCtl& k = ctl[q];
            std::memset(&k, 0, sizeof k);
            const double h3 = h->h * h->h * h->h;
            const double Q = op.beta * h->sum_w_in * h->h * h->h;
            k.tol = tol[q];
            k.tau = Q > 0 ? (double)h->n_fluid * h3 / Q : std::pow(h->nz * h->h, 2) / h->D;
            k.n_unknown = (double)h->n_fluid;
        }
        // Defects in double-float (as in a single mixed solve): the states are double-float
        // pairs during these cycles, and a lattice leaves them at its tol or, if that lies
        // below what double-float defects resolve, at 10 x tau 2^-44 max_c d_c. Then every
        // state is joined and checked in FP64; lattices still above their tol continue
        // with FP64 checks.
        b->df = true;
        for (int q = 0; q < n; ++q)
            ctl[q].tol = std::max(tol[q], 10.0 * ctl[q].tau * std::ldexp(1.0, -44) *
                                              (ops[q].cfl / ops[q].dt));
        int64_t df_cycles = 0;
        std::vector<int> cur0(n);
        for (int q = 0; q < n; ++q) {
            rfb_soc_handle* h = b->hs[q];
            cur0[q] = h->s_cur;
            try {
                ensure_L2F(h, ops[q]);
                df_begin(h, false);
                CK(h, cudaStreamSynchronize(h->stream));
            } catch (Fail f) {
                bset_err(b, "lattice %d: %s", q, h->err.c_str());
                throw;
            }
            BatchInst& I = insts[q];
            const size_t N = h->N;
            for (int f = 0; f < 6; ++f) I.K2.f[f] = h->d_L2F + f * N;
            I.K2.diag = h->d_L2F + 6 * N;
            I.K2.b = h->d_L2F + 7 * N;
            I.sdf[0] = h->d_sdf[0];
            I.sdf[1] = h->d_sdf[1];
            I.cur = 0;
        }
        BCK(b, cudaMemcpy(b->d_insts, insts.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice));
        BCK(b, cudaMemcpy(b->d_ctl, ctl.data(), n * sizeof(BatchCtl), cudaMemcpyHostToDevice));
        // tensor maps of the two-sweep passes (local steps; re-encoded every solve, since a
        // handle's own solves may have swapped its two correction buffers)
        bool tb_ok = local;
        for (int q = 0; q < n && tb_ok; ++q) tb_ok = tb_eligible(b->hs[q], true);
        if (tb_ok) {
            // per solve, on the batch's device (an attribute of the kernel in that
            // device's context; see tb_prepare)
            {
                BCK(b, cudaFuncSetAttribute(batch_tbd_kernel<3, 128>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            tbd_smem<3>()));
                BCK(b, cudaFuncSetAttribute(batch_tbd_kernel<4, 128>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            tbd_smem<4>()));
                BCK(b, cudaFuncSetAttribute(batch_tbd_kernel<3, 64>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            tbd_smem<3, 64>()));
            }
            for (int wide = 0; wide < 2; ++wide) {   // 72- then 136-column boxes
                const int bw = wide ? TB_BW : TBDGeom<64>::BW;
                std::vector<BatchTBD> tbd(n);
                for (int q = 0; q < n; ++q) {
                    rfb_soc_handle* h = b->hs[q];
                    BatchTBD& T = tbd[q];
                    std::memset(&T, 0, sizeof T);
                    try {
                        for (int p = 0; p < 2; ++p)
                            tb_encode(h, &T.td[p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                      insts[q].delta[p], h->nz, bw);
                        tb_encode(h, &T.tr, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_r32, h->nz, bw);
                        tb_encode(h, &T.tu, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_u32, h->nz, bw);
                        tb_encode(h, &T.tv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_v32, h->nz, bw);
                        tb_encode(h, &T.tw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_w32,
                                  h->nz + 1, bw);
                        tb_encode(h, &T.tt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h->d_dtc, h->nz, bw);
                    } catch (Fail f) {
                        bset_err(b, "lattice %d: %s", q, h->err.c_str());
                        throw;
                    }
                    T.nx = h->nx; T.ny = h->ny; T.nz = h->nz;
                    T.omc = (float)(1.0 - ops[q].cfl);
                    T.Dh = insts[q].C32.Dh;
                }
                BatchTBD*& dst = wide ? b->d_tbd : b->d_tbdn;
                if (!dst) BCK(b, cudaMalloc((void**)&dst, n * sizeof(BatchTBD)));
                BCK(b, cudaMemcpy(dst, tbd.data(), n * sizeof(BatchTBD), cudaMemcpyHostToDevice));
            }
            cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
        } else if (b->tb_nst) {
            b->tb_nst = 0;   // a global step: the one-sweep kernel (the graphs hold passes)
            if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
            if (b->loop_exec) { cudaGraphExecDestroy(b->loop_exec); b->loop_exec = nullptr; }
        }
        BCK(b, cudaMemsetAsync(b->d_tberr, 0, sizeof(unsigned int), b->stream));
        // opts.fp32_kernel: 0 the faster, 1 the one-sweep kernel, 2 two-sweep passes (tile
        // width, stages and chunk timed), 3 .. 6 passes with 128-column tiles, 7 / 8 passes
        // with 64-column tiles (mode 3 and 4 below)
        if (o.fp32_kernel > 8) {
            bset_err(b, "opts.fp32_kernel of a batch must be 0 .. 8");
            return RFB_ERR_INVALID_ARG;
        }
        const int k32 = o.fp32_kernel;
        const int mode = k32 <= 2 ? k32 : k32 <= 6 ? 3 : 4;
        if (mode >= 2 && !tb_ok) {
            bset_err(b, "two-sweep passes need local steps and nz >= 2 in every lattice");
            return RFB_ERR_INVALID_ARG;
        }
        if (!b->tuned_kchunk || b->tuned_mode != mode) {
            autotune(b, local, insts, mode);
            b->tuned_mode = mode;
        }
        else {
            build_items(b, b->tuned_kchunk);
            b->grid_blocks = std::max(1, std::min(b->tuned_grid, b->n_items));
        }
        int every = o.check_every > 0 ? std::max(2, o.check_every + (o.check_every & 1))
                                      : b->tuned_every;
        if (b->tb_nst) every = (every + 3) / 4 * 4;   // whole passes, result in delta[0]
        // residual of the starting states (forcing for the first cycle)
        batch_check(b, false, 0);
        BCK(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, n * sizeof(BatchCtl), cudaMemcpyDeviceToHost,
                               b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        int64_t done = 0;
        rfb_status st = RFB_OK;
        auto all_done = [&]() {
            for (int q = 0; q < n; ++q)
                if (!b->h_ctl[q].converged && !b->h_ctl[q].nonfinite) return false;
            return true;
        };
        int64_t graph_launches = 0;
        const bool device_loop = o.timeout_ms == 0;
        for (int phase = 0; phase < 2; ++phase) {
            // Without a timeout the cycles run in a device-driven loop (a conditional while
            // node): one graph launch runs up to 64 cycles and stops by itself once every
            // lattice has converged, so the host waits once per launch, not once per cycle.
            // A timeout needs the host between cycles: one captured cycle per launch.
            if (device_loop) {
                build_loop_graph(b, every, local);
            } else if (!b->exec || b->exec_every != every || b->exec_df != b->df) {
                if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
                cudaGraph_t g = nullptr;
                BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = b->launches;
                try {
                    batch_cycle(b, every, local);
                } catch (Fail) {
                    cudaStreamEndCapture(b->stream, &g);
                    if (g) cudaGraphDestroy(g);
                    throw;
                }
                b->launches = l0;   // counted when replayed
                BCK(b, cudaStreamEndCapture(b->stream, &g));
                BCK(b, cudaGraphInstantiate(&b->exec, g, 0));
                cudaGraphDestroy(g);
                b->exec_every = every;
                b->exec_df = b->df;
            }
            while (!all_done()) {
                if (done >= o.max_sweeps) { st = RFB_ERR_NOT_CONVERGED; break; }
                if (device_loop) {
                    const int64_t left = (o.max_sweeps - done + every - 1) / every;
                    BatchLoop lp{0, (int)std::min<int64_t>(64, left), n, 0};
                    *b->h_loop = lp;
                    BCK(b, cudaMemcpyAsync(b->d_loop, b->h_loop, sizeof(BatchLoop),
                                           cudaMemcpyHostToDevice, b->stream));
                    BCK(b, cudaGraphLaunch(b->loop_exec, b->stream));
                    BCK(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, n * sizeof(BatchCtl),
                                           cudaMemcpyDeviceToHost, b->stream));
                    BCK(b, cudaMemcpyAsync(b->h_loop, b->d_loop, sizeof(BatchLoop),
                                           cudaMemcpyDeviceToHost, b->stream));
                    BCK(b, cudaStreamSynchronize(b->stream));
                    const int cyc = b->h_loop->cycles;
                    b->launches += (int64_t)cyc * (every + 4);
                    done += (int64_t)cyc * every;
                    ++graph_launches;
                    if (cyc < 1) {
                        bset_err(b, "the device-driven batch loop ran no cycle");
                        throw Fail{RFB_ERR_CUDA};
                    }
                    continue;
                }
                if (o.timeout_ms > 0 && std::chrono::duration<double, std::milli>(
                                            std::chrono::steady_clock::now() - t0).count() >= o.timeout_ms) {
                    bset_err(b, "opts.timeout_ms reached after %lld sweeps", (long long)done);
                    st = RFB_ERR_NOT_CONVERGED;
                    break;
                }
                BCK(b, cudaGraphLaunch(b->exec, b->stream));
                b->launches += every + 3;
                BCK(b, cudaStreamSynchronize(b->stream));
                done += every;
                ++graph_launches;
            }
            if (!b->df) break;
            df_cycles = done / every;
            // double-float phase over: join every state, then check in FP64 against the
            // lattice's own tol (lattices that left the phase are checked again; any above
            // their tol continue with FP64 checks)
            BCK(b, cudaMemcpy(insts.data(), b->d_insts, n * sizeof(BatchInst),
                              cudaMemcpyDeviceToHost));
            for (int q = 0; q < n; ++q) {
                rfb_soc_handle* h = b->hs[q];
                join64_kernel<<<flat_grid(h->N), 256, 0, b->stream>>>(
                    h->d_sdf[insts[q].cur], h->d_s[cur0[q]], h->N);
                BLAUNCHED(b);
                insts[q].cur = cur0[q];
                b->h_ctl[q].tol = tol[q];
                if (b->h_ctl[q].converged) {
                    insts[q].active = 1;
                    b->h_ctl[q].converged = 0;
                }
            }
            BCK(b, cudaMemcpyAsync(b->d_insts, insts.data(), n * sizeof(BatchInst),
                                   cudaMemcpyHostToDevice, b->stream));
            BCK(b, cudaMemcpyAsync(b->d_ctl, b->h_ctl, n * sizeof(BatchCtl),
                                   cudaMemcpyHostToDevice, b->stream));
            b->df = false;
            batch_check(b, false, 0);
            BCK(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, n * sizeof(BatchCtl),
                                   cudaMemcpyDeviceToHost, b->stream));
            BCK(b, cudaStreamSynchronize(b->stream));
            if (st != RFB_OK) break;
        }
        BCK(b, cudaMemcpy(insts.data(), b->d_insts, n * sizeof(BatchInst), cudaMemcpyDeviceToHost));
        unsigned int tb_bad = 0;
        BCK(b, cudaMemcpy(&tb_bad, b->d_tberr, sizeof tb_bad, cudaMemcpyDeviceToHost));
        if (tb_bad) {
            bset_err(b, "a TMA stage of the batched two-sweep pass did not arrive in time");
            st = RFB_ERR_CUDA;
        }
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        for (int q = 0; q < n; ++q) {
            rfb_soc_handle* h = b->hs[q];
            h->s_cur = insts[q].cur;
            h->have_state = true;
            h->s_converged = b->h_ctl[q].converged != 0;
            if (b->h_ctl[q].nonfinite) st = RFB_ERR_NONFINITE;
            if (res) {
                rfb_solve_result r{};
                fill_result(h, ops[q], &r, h->n_fluid, b->h_ctl[q].sums);
                r.residual = b->h_ctl[q].residual;
                r.sweeps = b->h_ctl[q].sweeps;
                r.time_ms = ms;
                res[q] = r;
            }
        }
        if (info) {
            info->kchunk = b->tuned_kchunk;
            info->sweeps_per_cycle = every;
            info->n_items = b->n_items;
            info->grid_blocks = b->grid_blocks;
            info->sweep_ms = b->tuned_sweep_ms;
            info->check_ms = b->tuned_check_ms;
            info->cycles = done / every;
            info->graph_launches = graph_launches;
            info->pass_stages = b->tb_nst;
            info->pass_chunk = b->tb_nst ? b->tb_lc : 0;
            info->pass_tile_cols = b->tb_nst ? b->tb_txi : 0;
            info->df_cycles = (int32_t)df_cycles;
            info->time_ms = ms;
            info->launches = b->launches;
        }
        return st;
    } catch (Fail f) {
        return f.st;
    }
}

}  // extern "C"

extern "C" rfb_status rfb_soc_batch_set_stream(rfb_batch* b, void* stream) {
    if (!b) return RFB_ERR_INVALID_ARG;
    b->err.clear();
    if (stream == nullptr || stream == (void*)cudaStreamLegacy ||
        stream == (void*)cudaStreamPerThread) {
        bset_err(b, "a batch needs a created stream (its cycle is captured into a CUDA graph)");
        return RFB_ERR_INVALID_ARG;
    }
    try {
        BCK(b, cudaSetDevice(b->device));
        BCK(b, cudaStreamSynchronize(b->stream));
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->loop_exec) { cudaGraphExecDestroy(b->loop_exec); b->loop_exec = nullptr; }
        if (b->own_stream) { cudaStreamDestroy(b->stream); b->own_stream = false; }
        b->stream = (cudaStream_t)stream;
    } catch (Fail f) {
        return f.st;
    }
    return RFB_OK;
}
