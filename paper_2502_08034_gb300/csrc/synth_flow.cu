// Potential-flow fixture on the GPU (input generation for benchmarks and tests; not part
// of the state-of-charge solver and not called by it).
//
// Discrete potential flow on the fluid cells of a voxel lattice: phi = 1 on inlet faces
// (low-z face of plane 0), phi = 0 on outlet faces (high-z face of plane nz-1), no flux
// through fiber faces and side walls. Cell-to-cell conductance 1, cell-to-face 2.
// Unknown: psi = phi - phi_lin with phi_lin = 1 - (k + 1/2)/nz, so that the rounding
// floor of the face differences is set by |psi| << 1. Jacobi-preconditioned FP64 CG,
// deterministic (fixed-order block reductions), no host synchronisation inside the
// iteration except every `check_every` iterations for the true residual.
// Face velocities u = -grad(phi) are then scaled so that the mean of W over fluid
// z-faces (inlet and outlet faces included) equals u_mean.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

namespace {

constexpr int TPB = 256;
constexpr int NB = 152 * 8;   // reduction blocks (grid-stride)

struct G {
    int nx, ny, nz;
    int64_t N, nxny;
    const uint8_t* solid;
};

__device__ __forceinline__ bool fl(const G& g, int64_t c) { return !g.solid[c]; }

// (A x)_c for fluid c
__device__ __forceinline__ double apply_row(const G& g, const double* x, int64_t c, int i, int j,
                                            int k) {
    const double xc = x[c];
    double a = 0.0;
    if (i > 0 && fl(g, c - 1)) a += xc - x[c - 1];
    if (i + 1 < g.nx && fl(g, c + 1)) a += xc - x[c + 1];
    if (j > 0 && fl(g, c - g.nx)) a += xc - x[c - g.nx];
    if (j + 1 < g.ny && fl(g, c + g.nx)) a += xc - x[c + g.nx];
    if (k > 0 && fl(g, c - g.nxny)) a += xc - x[c - g.nxny];
    if (k + 1 < g.nz && fl(g, c + g.nxny)) a += xc - x[c + g.nxny];
    if (k == 0) a += 2.0 * xc;
    if (k == g.nz - 1) a += 2.0 * xc;
    return a;
}

// b - A phi_lin, exactly: phi_lin differs by dl = 1/nz between z neighbours, by 0 along
// x and y, and by dl/2 from the inlet value 1 and the outlet value 0.
__device__ __forceinline__ double rhs_lin(const G& g, int64_t c, int k) {
    const double dl = 1.0 / g.nz;
    double t = 0.0;
    if (k > 0 && fl(g, c - g.nxny)) t += 1.0;
    if (k + 1 < g.nz && fl(g, c + g.nxny)) t -= 1.0;
    if (k == 0) t += 1.0;
    if (k == g.nz - 1) t -= 1.0;
    return t * dl;
}

__device__ __forceinline__ double diag_of(const G& g, int64_t c, int i, int j, int k) {
    double d = 0.0;
    if (i > 0 && fl(g, c - 1)) d += 1.0;
    if (i + 1 < g.nx && fl(g, c + 1)) d += 1.0;
    if (j > 0 && fl(g, c - g.nx)) d += 1.0;
    if (j + 1 < g.ny && fl(g, c + g.nx)) d += 1.0;
    if (k > 0 && fl(g, c - g.nxny)) d += 1.0;
    if (k + 1 < g.nz && fl(g, c + g.nxny)) d += 1.0;
    if (k == 0) d += 2.0;
    if (k == g.nz - 1) d += 2.0;
    return d;
}

__device__ __forceinline__ void decompose(const G& g, int64_t c, int& i, int& j, int& k) {
    i = (int)(c % g.nx);
    j = (int)((c / g.nx) % g.ny);
    k = (int)(c / g.nxny);
}

__device__ double block_sum(double v) {
    __shared__ double sh[TPB / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < TPB / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}

__device__ double block_max(double v) {
    __shared__ double sh[TPB / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < TPB / 32; ++w) r = fmax(r, sh[w]);
    __syncthreads();
    return r;
}

// rhs = b - A phi_lin ; x = 0 ; r = rhs ; z = r / diag ; p = z ; partial r.z
__global__ void k_init(G g, double* rhs, double* x, double* r, double* z, double* p,
                       double* dinv, double* part) {
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)TPB + threadIdx.x; c < g.N;
         c += (int64_t)gridDim.x * TPB) {
        double rv = 0.0, di = 0.0;
        if (fl(g, c)) {
            int i, j, k;
            decompose(g, c, i, j, k);
            rv = rhs_lin(g, c, k);
            double d = diag_of(g, c, i, j, k);
            di = d > 0 ? 1.0 / d : 0.0;
        }
        rhs[c] = rv;
        x[c] = 0.0;
        r[c] = rv;
        dinv[c] = di;
        z[c] = rv * di;
        p[c] = rv * di;
        acc += rv * rv * di;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_finalize(const double* part, int n, double* out) {
    __shared__ double sh[TPB];
    double a = 0.0;
    for (int b = threadIdx.x; b < n; b += TPB) a += part[b];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_finalize_max(const double* part, int n, double* out) {
    __shared__ double sh[TPB];
    double a = 0.0;
    for (int b = threadIdx.x; b < n; b += TPB) a = fmax(a, part[b]);
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// q = A p ; partial p.q
__global__ void k_matvec(G g, const double* p, double* q, double* part) {
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)TPB + threadIdx.x; c < g.N;
         c += (int64_t)gridDim.x * TPB) {
        double a = 0.0;
        if (fl(g, c)) {
            int i, j, k;
            decompose(g, c, i, j, k);
            a = apply_row(g, p, c, i, j, k);
        }
        q[c] = a;
        acc += p[c] * a;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// alpha = rz / pq ; x += alpha p ; r -= alpha q ; z = dinv r ; partial r.z
__global__ void k_update(int64_t N, const double* sc, double* x, double* r, double* z,
                         const double* p, const double* q, const double* dinv, double* part) {
    const double alpha = sc[0] / sc[1];
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)TPB + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * TPB) {
        x[c] += alpha * p[c];
        const double rv = r[c] - alpha * q[c];
        r[c] = rv;
        const double zv = dinv[c] * rv;
        z[c] = zv;
        acc += rv * zv;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// beta = rz_new / rz ; p = z + beta p  (the host then copies rz_new over rz)
__global__ void k_pupdate(int64_t N, const double* rz_old, const double* rz_new, double* p,
                          const double* z) {
    const double beta = rz_new[0] / rz_old[0];
    for (int64_t c = blockIdx.x * (int64_t)TPB + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * TPB)
        p[c] = z[c] + beta * p[c];
}

// true residual max | rhs - A x | over fluid cells
__global__ void k_true_res(G g, const double* rhs, const double* x, double* part) {
    double m = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)TPB + threadIdx.x; c < g.N;
         c += (int64_t)gridDim.x * TPB) {
        if (fl(g, c)) {
            int i, j, k;
            decompose(g, c, i, j, k);
            m = fmax(m, fabs(rhs[c] - apply_row(g, x, c, i, j, k)));
        }
    }
    m = block_max(m);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// face velocities (unscaled, times h): U (nz, ny, nx+1), V (nz, ny+1, nx), W (nz+1, ny, nx)
__global__ void k_faces(G g, const double* x, double* U, double* V, double* W, double* part,
                        double* part_cnt) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const double dl = 1.0 / nz;   // phi_lin(k) - phi_lin(k+1)
    double sw = 0.0, cnt = 0.0;
    const int64_t nU = (int64_t)(nx + 1) * ny * nz;
    const int64_t nV = (int64_t)nx * (ny + 1) * nz;
    const int64_t nW = (int64_t)nx * ny * (nz + 1);
    for (int64_t q = blockIdx.x * (int64_t)TPB + threadIdx.x; q < nU + nV + nW;
         q += (int64_t)gridDim.x * TPB) {
        if (q < nU) {
            const int a = (int)(q % (nx + 1));
            const int64_t rest = q / (nx + 1);
            const int j = (int)(rest % ny), k = (int)(rest / ny);
            double v = 0.0;
            if (a > 0 && a < nx) {
                const int64_t c0 = (a - 1) + (int64_t)nx * j + g.nxny * k;
                if (fl(g, c0) && fl(g, c0 + 1)) v = -(x[c0 + 1] - x[c0]);
            }
            U[q] = v;
        } else if (q < nU + nV) {
            const int64_t qq = q - nU;
            const int i = (int)(qq % nx);
            const int64_t rest = qq / nx;
            const int b = (int)(rest % (ny + 1)), k = (int)(rest / (ny + 1));
            double v = 0.0;
            if (b > 0 && b < ny) {
                const int64_t c0 = i + (int64_t)nx * (b - 1) + g.nxny * k;
                if (fl(g, c0) && fl(g, c0 + nx)) v = -(x[c0 + nx] - x[c0]);
            }
            V[qq] = v;
        } else {
            const int64_t qq = q - nU - nV;
            const int64_t ij = qq % g.nxny;
            const int k = (int)(qq / g.nxny);
            double v = 0.0;
            bool face = false;
            if (k == 0) {
                // phi <= 1 in the exact solution, so inflow is >= 0; a negative value
                // here is CG rounding in a stagnant pocket
                if (fl(g, ij)) { v = fmax(dl - 2.0 * x[ij], 0.0); face = true; }
            } else if (k == nz) {
                const int64_t c = ij + g.nxny * (nz - 1);
                if (fl(g, c)) { v = fmax(dl + 2.0 * x[c], 0.0); face = true; }
            } else {
                const int64_t c0 = ij + g.nxny * (k - 1);
                if (fl(g, c0) && fl(g, c0 + g.nxny)) {
                    v = dl - (x[c0 + g.nxny] - x[c0]);
                    face = true;
                }
            }
            W[qq] = v;
            if (face) { sw += v; cnt += 1.0; }
        }
    }
    sw = block_sum(sw);
    if (threadIdx.x == 0) part[blockIdx.x] = sw;
    cnt = block_sum(cnt);
    if (threadIdx.x == 0) part_cnt[blockIdx.x] = cnt;
}

__global__ void k_scale(double* a, int64_t n, const double* sw, const double* cnt, double u_mean) {
    const double s = u_mean / (sw[0] / cnt[0]);
    for (int64_t q = blockIdx.x * (int64_t)TPB + threadIdx.x; q < n; q += (int64_t)gridDim.x * TPB)
        a[q] *= s;
}

// max over fluid cells of |sum of outward face velocities| (scaled arrays)
__global__ void k_div(G g, const double* U, const double* V, const double* W, double* part) {
    double m = 0.0;
    const int nx = g.nx, ny = g.ny;
    for (int64_t c = blockIdx.x * (int64_t)TPB + threadIdx.x; c < g.N;
         c += (int64_t)gridDim.x * TPB) {
        if (!fl(g, c)) continue;
        const int i = (int)(c % nx);
        const int64_t rest = c / nx;
        const int j = (int)(rest % ny), k = (int)(rest / ny);
        const int64_t u0 = i + (int64_t)(nx + 1) * (j + (int64_t)ny * k);
        const int64_t v0 = i + (int64_t)nx * (j + (int64_t)(ny + 1) * k);
        const int64_t w0 = c;
        const double d = (U[u0 + 1] - U[u0]) + (V[v0 + nx] - V[v0]) + (W[w0 + g.nxny] - W[w0]);
        m = fmax(m, fabs(d));
    }
    m = block_max(m);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

}  // namespace

extern "C" {

// Returns 0 on success, 1 on bad arguments, 2 on a CUDA error, 3 if the CG did not reach
// the tolerance (the best fields found are still written). info (host, 4 doubles):
// iterations, max|div u| / u_mean, true residual / (mean unscaled W), superficial q.
int rfb_synth_potential_flow(int nx, int ny, int nz, double h, double u_mean, double tol,
                             int max_iter, int check_every, const uint8_t* d_solid,
                             double* d_U, double* d_V, double* d_W, double* info,
                             void* stream_) {
    if (nx < 1 || ny < 1 || nz < 2 || !(h > 0) || !(u_mean > 0) || !d_solid || !d_U || !d_V ||
        !d_W || !info || check_every < 1)
        return 1;
    cudaStream_t st = (cudaStream_t)stream_;
    G g{nx, ny, nz, (int64_t)nx * ny * nz, (int64_t)nx * ny, d_solid};
    const int64_t N = g.N;
    double *rhs = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
           *dinv = nullptr, *part = nullptr, *part2 = nullptr, *sc = nullptr;
    double* hs = nullptr;
    int rc = 0;
#define FCK(call) do { if ((call) != cudaSuccess) { rc = 2; goto done; } } while (0)
    FCK(cudaMalloc(&rhs, N * 8)); FCK(cudaMalloc(&x, N * 8)); FCK(cudaMalloc(&r, N * 8));
    FCK(cudaMalloc(&z, N * 8)); FCK(cudaMalloc(&p, N * 8)); FCK(cudaMalloc(&q, N * 8));
    FCK(cudaMalloc(&dinv, N * 8)); FCK(cudaMalloc(&part, NB * 8)); FCK(cudaMalloc(&part2, NB * 8));
    // scalars: 0 rz, 1 pq, 2 rz_new, 3 max true residual, 4 sum W, 5 face count, 6 div
    FCK(cudaMalloc(&sc, 8 * 8));
    FCK(cudaMallocHost(&hs, 8 * 8));
    {
        k_init<<<NB, TPB, 0, st>>>(g, rhs, x, r, z, p, dinv, part);
        k_finalize<<<1, TPB, 0, st>>>(part, NB, sc + 0);
        int it = 0;
        double best = INFINITY;
        int since_best = 0;
        double wmean = 1.0 / nz;   // refined below from the actual faces
        bool converged = false;
        while (it < max_iter) {
            for (int s = 0; s < check_every && it < max_iter; ++s, ++it) {
                k_matvec<<<NB, TPB, 0, st>>>(g, p, q, part);
                k_finalize<<<1, TPB, 0, st>>>(part, NB, sc + 1);
                k_update<<<NB, TPB, 0, st>>>(N, sc, x, r, z, p, q, dinv, part);
                k_finalize<<<1, TPB, 0, st>>>(part, NB, sc + 2);
                k_pupdate<<<NB, TPB, 0, st>>>(N, sc + 0, sc + 2, p, z);
                FCK(cudaMemcpyAsync(sc + 0, sc + 2, 8, cudaMemcpyDeviceToDevice, st));
            }
            k_true_res<<<NB, TPB, 0, st>>>(g, rhs, x, part);
            k_finalize_max<<<1, TPB, 0, st>>>(part, NB, sc + 3);
            k_faces<<<NB, TPB, 0, st>>>(g, x, d_U, d_V, d_W, part, part2);
            k_finalize<<<1, TPB, 0, st>>>(part, NB, sc + 4);
            k_finalize<<<1, TPB, 0, st>>>(part2, NB, sc + 5);
            FCK(cudaMemcpyAsync(hs, sc, 8 * 8, cudaMemcpyDeviceToHost, st));
            FCK(cudaStreamSynchronize(st));
            wmean = hs[4] / hs[5];
            const double achieved = hs[3] / wmean;
            info[2] = achieved;
            if (achieved < 0.5 * tol) { converged = true; break; }
            if (achieved < 0.7 * best) { best = achieved; since_best = 0; }
            else if (++since_best >= 20) break;   // stagnated at the rounding floor
        }
        info[0] = it;
        // faces from the final iterate, scaled to the requested mean
        k_faces<<<NB, TPB, 0, st>>>(g, x, d_U, d_V, d_W, part, part2);
        k_finalize<<<1, TPB, 0, st>>>(part, NB, sc + 4);
        k_finalize<<<1, TPB, 0, st>>>(part2, NB, sc + 5);
        const int64_t nU = (int64_t)(nx + 1) * ny * nz, nV = (int64_t)nx * (ny + 1) * nz,
                      nW = (int64_t)nx * ny * (nz + 1);
        k_scale<<<NB, TPB, 0, st>>>(d_U, nU, sc + 4, sc + 5, u_mean);
        k_scale<<<NB, TPB, 0, st>>>(d_V, nV, sc + 4, sc + 5, u_mean);
        k_scale<<<NB, TPB, 0, st>>>(d_W, nW, sc + 4, sc + 5, u_mean);
        k_div<<<NB, TPB, 0, st>>>(g, d_U, d_V, d_W, part);
        k_finalize_max<<<1, TPB, 0, st>>>(part, NB, sc + 6);
        FCK(cudaMemcpyAsync(hs, sc, 8 * 8, cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        FCK(cudaGetLastError());
        info[1] = hs[6] / u_mean;
        {
            // superficial velocity: sum of inlet W / (nx ny), from the scaled W
            std::vector<double> w0(g.nxny);
            FCK(cudaMemcpy(w0.data(), d_W, g.nxny * 8, cudaMemcpyDeviceToHost));
            double s = 0.0;
            for (double v : w0) s += v;
            info[3] = s / (double)g.nxny;
        }
        if (!converged && !(info[1] < tol)) rc = 3;
    }
done:
    cudaFree(rhs); cudaFree(x); cudaFree(r); cudaFree(z); cudaFree(p); cudaFree(q);
    cudaFree(dinv); cudaFree(part); cudaFree(part2); cudaFree(sc);
    if (hs) cudaFreeHost(hs);
#undef FCK
    (void)h;
    return rc;
}

}  // extern "C"
