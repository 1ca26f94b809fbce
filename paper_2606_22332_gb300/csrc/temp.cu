// temp.cu -- the TemperatureGrid sensor (Appendix "TemperatureGrid Sensor
// Model") and the contact-area estimate of its conduction term, behind the
// tg_temp_* / tg_contact_area entry points of include/tg.h.
//
// One CTA per grid holds the grid in shared memory (rows of the z axis padded
// by one float, so that a warp's reads down any axis fall in distinct banks)
// and runs the whole step there:
//  1. diffusion: mirror padding to twice the size on every axis followed by a
//     real FFT, a per-mode division by 1 + alpha dt k^2 and the inverse FFT
//     cropped back to the grid is the orthonormal DCT-II of the grid, the same
//     division per mode (k_m = pi m / (n d) on each axis), and the inverse
//     DCT.  Each transform is three contractions with an n x n matrix, one
//     per axis; a thread forms four outputs of one (line, column) pair per
//     pass (the sides are powers of two: indices split by shifts).  The field is transformed relative to its first cell's value,
//     which comes back through the zero mode's factor.
//  2. source: T += dt q / (dz rho c_p);
//  3. contact conduction: every contact of the grid adds
//     dt k_eff (T_other - T_c) (A / V)^2 / (rho c_p) to its cell, all from the
//     field after the source (k_eff = 2 k k_b / (k + k_b));
//  4. radiation and convection on the cells of the grid's faces:
//     T -= dt (eps sigma (T_K^4 - T_amb,K^4) + h (T - T_amb)) / (rho c_p), the
//     fourth-power difference formed as (T_K - T_a)(T_K + T_a)(T_K^2 + T_a^2);
//  5. the measured readout's lag: T_meas += dt / tau (T - T_meas), or
//     T_meas = T for tau <= 0.
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace tg {

constexpr int kTempThreads = 256;
constexpr int kTempMaxN = 32;
constexpr int kTempMaxPadded = 12288;  // nx * ny * (nz + 1) floats per grid buffer

struct TempArgs {
    int G, nx, ny, nz;
    int lx, ly, lz;           // log2 of the sides (powers of two)
    const float* voxel;       // [G][3]
    const float* material;    // [G][7]: k, rho, c_p, emissivity, h, tau, base
    const float* dct;         // C_x, C_x^T, C_y, C_y^T, C_z, C_z^T (n x n each, row-major)
    float k2_floor;
    float dt, t_amb;
    const float* source;      // [G][cells] or null
    int n_contacts;
    const int32_t* c_off;     // [G + 1] or null
    const int32_t* c_cell;
    const float* c_temp;
    const float* c_k;
    const float* c_area;
    float* T;                 // [G][cells]
    float* Tm;                // [G][cells]
};

// dst(p, m, q) = sum_j W(m, j) src(p, j, q), with Wt[j][m] = W(m, j) (N x N),
// over a [P][N][Q] view with element strides (sp, sj, sq); P and Q powers of
// two (lP, lQ their logs); the contraction unrolled over its length N
template <int N>
__device__ __forceinline__ void temp_contract_n(const float* __restrict__ src, float* __restrict__ dst,
                                                const float* __restrict__ Wt, int lP, int lQ, int sp, int sj, int sq) {
    constexpr int nb = N / 4, lnb = N == 4 ? 0 : N == 8 ? 1 : N == 16 ? 2 : 3;
    const int work = 1 << (lP + lnb + lQ);
    for (int t = threadIdx.x; t < work; t += kTempThreads) {
        // lanes run over q, then p
        const int q = t & ((1 << lQ) - 1), r = t >> lQ, p = r & ((1 << lP) - 1), mb = r >> lP;
        const float* s = src + p * sp + q * sq;
        const float4* w = reinterpret_cast<const float4*>(Wt) + mb;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float v = s[j * sj];
            const float4 c = w[j * nb];
            acc.x = fmaf(c.x, v, acc.x);
            acc.y = fmaf(c.y, v, acc.y);
            acc.z = fmaf(c.z, v, acc.z);
            acc.w = fmaf(c.w, v, acc.w);
        }
        float* d = dst + p * sp + q * sq + (4 * mb) * sj;
        d[0] = acc.x;
        d[sj] = acc.y;
        d[2 * sj] = acc.z;
        d[3 * sj] = acc.w;
    }
}

__device__ __forceinline__ void temp_contract(const float* __restrict__ src, float* __restrict__ dst,
                                              const float* __restrict__ Wt, int lP, int ln, int lQ, int sp, int sj,
                                              int sq) {
    switch (ln) {
    case 2: temp_contract_n<4>(src, dst, Wt, lP, lQ, sp, sj, sq); break;
    case 3: temp_contract_n<8>(src, dst, Wt, lP, lQ, sp, sj, sq); break;
    case 4: temp_contract_n<16>(src, dst, Wt, lP, lQ, sp, sj, sq); break;
    default: temp_contract_n<32>(src, dst, Wt, lP, lQ, sp, sj, sq); break;
    }
}

__global__ void __launch_bounds__(kTempThreads) temp_step_kernel(const TempArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int g = blockIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz, SZ = nz + 1, lx = a.lx, ly = a.ly, lz = a.lz;
    const int cells = nx * ny * nz, padded = nx * ny * SZ;
    float* A = sm;
    float* B = sm + padded;
    float* W = B + padded;  // the six matrices
    const int wx = nx * nx, wy = ny * ny, wz = nz * nz;
    for (int i = threadIdx.x; i < 2 * (wx + wy + wz); i += kTempThreads) W[i] = a.dct[i];
    const float* Cx = W;            // rows m, columns i: C_x(m, i)
    const float* CxT = W + wx;      // CxT[i][m] = C_x(m, i)
    const float* Cy = CxT + wx;
    const float* CyT = Cy + wy;
    const float* Cz = CyT + wy;
    const float* CzT = Cz + wz;
    const float* Tg = a.T + (size_t)g * cells;
    const float c0 = __ldg(Tg);
    for (int e = threadIdx.x; e < cells; e += kTempThreads) A[(e >> lz) * SZ + (e & (nz - 1))] = Tg[e] - c0;
    __syncthreads();
    // forward DCT-II on z, y, x (the matrix's transpose is the operand of the contraction)
    temp_contract(A, B, CzT, lx + ly, lz, 0, SZ, 1, 0);
    __syncthreads();
    temp_contract(B, A, CyT, lx, ly, lz, ny * SZ, SZ, 1);
    __syncthreads();
    temp_contract(A, B, CxT, ly, lx, lz, SZ, ny * SZ, 1);
    __syncthreads();
    // per-mode implicit step
    const float* vox = a.voxel + 3 * g;
    const float* mat = a.material + 7 * g;
    const float kc = mat[0], rc = mat[1] * mat[2];
    const float adt = a.dt * (kc / rc);
    {
        const float px = 3.14159265358979f / (nx * vox[0]), py = 3.14159265358979f / (ny * vox[1]),
                    pz = 3.14159265358979f / (nz * vox[2]);
        for (int e = threadIdx.x; e < cells; e += kTempThreads) {
            const int mz = e & (nz - 1), r = e >> lz, my = r & (ny - 1), mx = r >> ly;
            const float kx = mx * px, ky = my * py, kz = mz * pz;
            const float k2 = fmaxf(fmaf(kx, kx, fmaf(ky, ky, kz * kz)), a.k2_floor);
            B[r * SZ + mz] *= __frcp_rn(fmaf(adt, k2, 1.0f));
        }
    }
    __syncthreads();
    // inverse DCT on x, y, z (the matrix itself is the operand)
    temp_contract(B, A, Cx, ly, lx, lz, SZ, ny * SZ, 1);
    __syncthreads();
    temp_contract(A, B, Cy, lx, ly, lz, ny * SZ, SZ, 1);
    __syncthreads();
    temp_contract(B, A, Cz, lx + ly, lz, 0, SZ, 1, 0);
    __syncthreads();
    const float base = c0 / fmaf(adt, a.k2_floor, 1.0f);  // the subtracted value through the zero mode
    const float* q = a.source ? a.source + (size_t)g * cells : nullptr;
    const float sq = a.dt / (vox[2] * rc);
    for (int e = threadIdx.x; e < cells; e += kTempThreads) {
        const int s = (e >> lz) * SZ + (e & (nz - 1));
        float t = A[s] + base;
        if (q) t = fmaf(sq, q[e], t);
        A[s] = t;
        B[s] = 0.0f;
    }
    __syncthreads();
    // contact conduction: every contact reads the field after the source; changes add
    if (a.c_off) {
        // device arrays are not checked on the host: clamp the range, skip cells out of range
        const int c_begin = min(max(a.c_off[g], 0), a.n_contacts), c_end = min(max(a.c_off[g + 1], 0), a.n_contacts);
        if (c_end > c_begin) {
            const float V = vox[0] * vox[1] * vox[2];
            for (int c = c_begin + threadIdx.x; c < c_end; c += kTempThreads) {
                const int cell = a.c_cell[c];
                if (cell < 0 || cell >= cells) continue;
                const int s = (cell >> lz) * SZ + (cell & (nz - 1));
                const float kb = a.c_k[c], av = a.c_area[c] / V;
                const float keff = 2.0f * kc * kb / (kc + kb);
                atomicAdd(&B[s], a.dt * keff * (a.c_temp[c] - A[s]) * av * av / rc);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < cells; e += kTempThreads) {
                const int s = (e >> lz) * SZ + (e & (nz - 1));
                A[s] += B[s];
            }
        }
    }
    // radiation and convection on the face cells, the lag, and the stores
    const float em = mat[3] * 5.670e-8f, h = mat[4], tau = mat[5];
    const float ta = a.t_amb, taK = ta + 273.15f;
    float* Tout = a.T + (size_t)g * cells;
    float* Tm = a.Tm + (size_t)g * cells;
    for (int e = threadIdx.x; e < cells; e += kTempThreads) {
        const int k = e & (nz - 1), r = e >> lz, j = r & (ny - 1), i = r >> ly;
        const int s = r * SZ + k;
        float t = A[s];
        if (i == 0 || i == nx - 1 || j == 0 || j == ny - 1 || k == 0 || k == nz - 1) {
            const float tK = t + 273.15f, d = t - ta;
            const float rad = em * d * (tK + taK) * fmaf(tK, tK, taK * taK);
            t -= a.dt * fmaf(h, d, rad) / rc;
        }
        Tout[e] = t;
        const float m = Tm[e];
        Tm[e] = tau > 0.0f ? fmaf(a.dt / tau, t - m, m) : t;
    }
}

__global__ void temp_fill_kernel(float* T, float* Tm, const float* material, int G, int cells, const uint8_t* mask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G * cells) return;
    const int g = (int)(i / cells);
    if (mask && !mask[g]) return;
    T[i] = Tm[i] = material[7 * g + 6];
}

// one thread per manifold: best-fit plane (the covariance's least eigenvector
// by cyclic Jacobi rotations), polar order about the centroid, shoelace area;
// fewer than three points give a disk of radius delta; floored at pi (d_w delta)^2
__global__ void contact_area_kernel(const float* pts, const int32_t* npts, const float* depth, int n_pairs,
                                    int max_pts, float d_w, float* area) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int n = min(max(npts[p], 0), max_pts);
    const float* P = pts + (size_t)p * max_pts * 3;
    const float dl = depth[p];
    float out;
    if (n < 3) {
        out = 3.14159265358979f * dl * dl;
    } else {
        double c[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) c[a] += P[3 * i + a];
        for (int a = 0; a < 3; ++a) c[a] /= n;
        double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int i = 0; i < n; ++i) {
            const double d[3] = {P[3 * i] - c[0], P[3 * i + 1] - c[1], P[3 * i + 2] - c[2]};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[a][b] += d[a] * d[b];
        }
        double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int sweep = 0; sweep < 12; ++sweep) {
            for (int pq = 0; pq < 3; ++pq) {
                const int a = pq == 2 ? 1 : 0, b = pq == 0 ? 1 : 2;
                if (fabs(M[a][b]) < 1e-300) continue;
                const double th = 0.5 * atan2(2.0 * M[a][b], M[b][b] - M[a][a]);
                const double cs = cos(th), sn = sin(th);
                for (int k = 0; k < 3; ++k) {  // M <- M J
                    const double x = M[k][a], y = M[k][b];
                    M[k][a] = cs * x - sn * y;
                    M[k][b] = sn * x + cs * y;
                }
                for (int k = 0; k < 3; ++k) {  // M <- J^T M
                    const double x = M[a][k], y = M[b][k];
                    M[a][k] = cs * x - sn * y;
                    M[b][k] = sn * x + cs * y;
                }
                for (int k = 0; k < 3; ++k) {  // V <- V J
                    const double x = V[k][a], y = V[k][b];
                    V[k][a] = cs * x - sn * y;
                    V[k][b] = sn * x + cs * y;
                }
            }
        }
        int lo = 0;
        if (M[1][1] < M[lo][lo]) lo = 1;
        if (M[2][2] < M[lo][lo]) lo = 2;
        const double nrm[3] = {V[0][lo], V[1][lo], V[2][lo]};
        // an in-plane basis: u orthogonal to the normal, v = n x u
        double u[3] = {fabs(nrm[0]) < 0.9 ? 1.0 : 0.0, fabs(nrm[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        const double un = u[0] * nrm[0] + u[1] * nrm[1];
        for (int a = 0; a < 3; ++a) u[a] -= un * nrm[a];
        const double ul = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < 3; ++a) u[a] /= ul;
        const double v[3] = {nrm[1] * u[2] - nrm[2] * u[1], nrm[2] * u[0] - nrm[0] * u[2], nrm[0] * u[1] - nrm[1] * u[0]};
        double x[16], y[16], ang[16];
        for (int i = 0; i < n; ++i) {
            const double d[3] = {P[3 * i] - c[0], P[3 * i + 1] - c[1], P[3 * i + 2] - c[2]};
            x[i] = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
            y[i] = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
            ang[i] = atan2(y[i], x[i]);
        }
        for (int i = 1; i < n; ++i) {  // insertion sort by polar angle
            const double xa = x[i], ya = y[i], aa = ang[i];
            int k = i - 1;
            while (k >= 0 && ang[k] > aa) {
                x[k + 1] = x[k];
                y[k + 1] = y[k];
                ang[k + 1] = ang[k];
                --k;
            }
            x[k + 1] = xa;
            y[k + 1] = ya;
            ang[k + 1] = aa;
        }
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const int j = i + 1 == n ? 0 : i + 1;
            s += x[i] * y[j] - y[i] * x[j];
        }
        out = (float)(0.5 * fabs(s));
    }
    area[p] = fmaxf(out, 3.14159265358979f * (d_w * dl) * (d_w * dl));
}

}  // namespace tg

using namespace tg;

namespace {

thread_local std::string g_temp_error;

tg_status tfail(tg_status st, const std::string& m) {
    g_temp_error = m;
    return st;
}

tg_status tcuda(cudaError_t e, const char* what) {
    return tfail(e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define TCK(call)                                       \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) return tcuda(_e, #call); \
    } while (0)

bool t_is_dev(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// orthonormal DCT-II matrix of size n: C(m, i) = s_m cos(pi m (i + 1/2) / n)
void dct_matrix(int n, std::vector<float>& C, std::vector<float>& Ct) {
    C.assign((size_t)n * n, 0.f);
    Ct.assign((size_t)n * n, 0.f);
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < n; ++m)
        for (int i = 0; i < n; ++i) {
            const double s = m == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
            const double v = s * std::cos(pi * m * (i + 0.5) / n);
            C[(size_t)m * n + i] = (float)v;
            Ct[(size_t)i * n + m] = (float)v;
        }
}

}  // namespace

struct tg_temp {
    int G = 0, nx = 0, ny = 0, nz = 0;
    float k2_floor = 0.f;
    float* voxel = nullptr;     // [G][3]
    float* material = nullptr;  // [G][7]
    float* dct = nullptr;
    float* T = nullptr;
    float* Tm = nullptr;
    uint8_t* mask = nullptr;    // [G] staging of a reset mask
    // staging of host contact arrays (grown on demand)
    void* scratch = nullptr;
    size_t scratch_cap = 0;
    size_t smem = 0;
};

extern "C" {

tg_status tg_temp_create(const tg_temp_desc* d, tg_temp** out) {
    if (!d || !out) return tfail(TG_ERR_INVALID_ARG, "desc and out are required");
    *out = nullptr;
    auto dim_ok = [](int n) { return n >= 4 && n <= kTempMaxN && (n & (n - 1)) == 0; };
    if (d->n_grids < 1 || !dim_ok(d->nx) || !dim_ok(d->ny) || !dim_ok(d->nz) ||
        d->nx * d->ny * (d->nz + 1) > kTempMaxPadded)
        return tfail(TG_ERR_INVALID_ARG, "n_grids >= 1 and nx, ny, nz in {4, 8, 16, 32} with nx*ny*(nz+1) <= 12288");
    if (!d->voxel || !d->material || !(d->k2_floor >= 0.0) || !std::isfinite(d->k2_floor))
        return tfail(TG_ERR_INVALID_ARG, "voxel and material arrays and a finite k2_floor >= 0 are required");
    const int G = d->n_grids;
    for (int g = 0; g < G; ++g) {
        for (int a = 0; a < 3; ++a)
            if (!(d->voxel[3 * g + a] > 0.0f) || !std::isfinite(d->voxel[3 * g + a]))
                return tfail(TG_ERR_INVALID_ARG, "voxel sizes must be finite and > 0");
        const float* m = d->material + 7 * g;
        if (!(m[0] >= 0.0f) || !(m[1] > 0.0f) || !(m[2] > 0.0f) || !(m[3] >= 0.0f) || !(m[4] >= 0.0f))
            return tfail(TG_ERR_INVALID_ARG, "material needs k >= 0, rho > 0, c_p > 0, emissivity >= 0, h >= 0");
        for (int a = 0; a < 7; ++a)
            if (!std::isfinite(m[a])) return tfail(TG_ERR_INVALID_ARG, "material values must be finite");
    }
    tg_temp* t = new tg_temp();
    t->G = G;
    t->nx = d->nx;
    t->ny = d->ny;
    t->nz = d->nz;
    t->k2_floor = (float)d->k2_floor;
    const size_t cells = (size_t)d->nx * d->ny * d->nz;
    std::vector<float> dct, C, Ct;
    for (int n : {d->nx, d->ny, d->nz}) {
        dct_matrix(n, C, Ct);
        dct.insert(dct.end(), C.begin(), C.end());
        dct.insert(dct.end(), Ct.begin(), Ct.end());
    }
    auto undo = [&](cudaError_t e, const char* what) {
        tg_temp_destroy(t);
        return tcuda(e, what);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&t->voxel, sizeof(float) * 3 * G)) != cudaSuccess) return undo(e, "voxel alloc");
    if ((e = cudaMalloc(&t->material, sizeof(float) * 7 * G)) != cudaSuccess) return undo(e, "material alloc");
    if ((e = cudaMalloc(&t->dct, sizeof(float) * dct.size())) != cudaSuccess) return undo(e, "dct alloc");
    if ((e = cudaMalloc(&t->T, sizeof(float) * cells * G)) != cudaSuccess) return undo(e, "field alloc");
    if ((e = cudaMalloc(&t->Tm, sizeof(float) * cells * G)) != cudaSuccess) return undo(e, "field alloc");
    if ((e = cudaMalloc(&t->mask, G)) != cudaSuccess) return undo(e, "mask alloc");
    cudaMemcpy(t->voxel, d->voxel, sizeof(float) * 3 * G, cudaMemcpyHostToDevice);
    cudaMemcpy(t->material, d->material, sizeof(float) * 7 * G, cudaMemcpyHostToDevice);
    if ((e = cudaMemcpy(t->dct, dct.data(), sizeof(float) * dct.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return undo(e, "upload");
    t->smem = sizeof(float) * (2 * (size_t)d->nx * d->ny * (d->nz + 1) + dct.size());
    // per device, the limit only grows: grids created earlier keep launching
    if ((e = raise_smem_limit((const void*)temp_step_kernel, t->smem)) != cudaSuccess) return undo(e, "shared memory");
    const int64_t n = (int64_t)cells * G;
    temp_fill_kernel<<<(unsigned)((n + 255) / 256), 256>>>(t->T, t->Tm, t->material, G, (int)cells, nullptr);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return undo(e, "initial fill");
    *out = t;
    return TG_OK;
}

void tg_temp_destroy(tg_temp* t) {
    if (!t) return;
    cudaDeviceSynchronize();
    for (void* p : {(void*)t->voxel, (void*)t->material, (void*)t->dct, (void*)t->T, (void*)t->Tm, (void*)t->mask,
                    t->scratch})
        if (p) cudaFree(p);
    delete t;
}

tg_status tg_temp_reset(tg_temp* t, const uint8_t* grid_mask, tg_stream stream) {
    if (!t) return tfail(TG_ERR_INVALID_ARG, "grid is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t* m = nullptr;
    if (grid_mask) {
        TCK(cudaMemcpyAsync(t->mask, grid_mask, t->G, cudaMemcpyDefault, st));
        m = t->mask;
    }
    const int cells = t->nx * t->ny * t->nz;
    const int64_t n = (int64_t)cells * t->G;
    temp_fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t->T, t->Tm, t->material, t->G, cells, m);
    TCK(cudaGetLastError());
    return TG_OK;
}

tg_status tg_temp_set(tg_temp* t, const float* field, const float* measured, tg_stream stream) {
    if (!t || !field) return tfail(TG_ERR_INVALID_ARG, "grid and field are required");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * t->nx * t->ny * t->nz * t->G;
    TCK(cudaMemcpyAsync(t->T, field, bytes, cudaMemcpyDefault, st));
    TCK(cudaMemcpyAsync(t->Tm, measured ? measured : field, bytes, cudaMemcpyDefault, st));
    return TG_OK;
}

tg_status tg_temp_step(tg_temp* t, const tg_temp_inputs* in, tg_stream stream) {
    if (!t || !in) return tfail(TG_ERR_INVALID_ARG, "grid and inputs are required");
    if (!(in->dt > 0.0) || !std::isfinite(in->dt) || !std::isfinite(in->t_amb))
        return tfail(TG_ERR_INVALID_ARG, "dt must be finite and > 0, t_amb finite");
    if (in->n_contacts < 0 || (in->n_contacts > 0 && (!in->contact_offsets || !in->contact_cell || !in->contact_temp ||
                                                     !in->contact_k || !in->contact_area)))
        return tfail(TG_ERR_INVALID_ARG, "contacts need offsets, cells, temperatures, conductivities and areas");
    if (in->source && !t_is_dev(in->source)) return tfail(TG_ERR_INVALID_ARG, "source must be a device buffer");
    cudaStream_t st = (cudaStream_t)stream;
    TempArgs a{};
    a.G = t->G;
    a.nx = t->nx;
    a.ny = t->ny;
    a.nz = t->nz;
    a.lx = __builtin_ctz((unsigned)t->nx);
    a.ly = __builtin_ctz((unsigned)t->ny);
    a.lz = __builtin_ctz((unsigned)t->nz);
    a.voxel = t->voxel;
    a.material = t->material;
    a.dct = t->dct;
    a.k2_floor = t->k2_floor;
    a.dt = (float)in->dt;
    a.t_amb = (float)in->t_amb;
    a.source = in->source;
    a.T = t->T;
    a.Tm = t->Tm;
    a.n_contacts = in->n_contacts;
    if (in->n_contacts > 0) {
        const size_t C = (size_t)in->n_contacts, G1 = (size_t)t->G + 1;
        const bool dev = t_is_dev(in->contact_offsets) && t_is_dev(in->contact_cell) && t_is_dev(in->contact_temp) &&
                         t_is_dev(in->contact_k) && t_is_dev(in->contact_area);
        if (dev) {
            a.c_off = in->contact_offsets;
            a.c_cell = in->contact_cell;
            a.c_temp = in->contact_temp;
            a.c_k = in->contact_k;
            a.c_area = in->contact_area;
        } else {
            // host arrays: checked here, then staged (the copies are ordered on the stream)
            const int cells = t->nx * t->ny * t->nz;
            if (in->contact_offsets[0] != 0 || in->contact_offsets[t->G] != in->n_contacts)
                return tfail(TG_ERR_INVALID_ARG, "contact_offsets must run from 0 to n_contacts");
            for (int g = 0; g < t->G; ++g)
                if (in->contact_offsets[g + 1] < in->contact_offsets[g])
                    return tfail(TG_ERR_INVALID_ARG, "contact_offsets must not decrease");
            for (size_t c = 0; c < C; ++c)
                if (in->contact_cell[c] < 0 || in->contact_cell[c] >= cells || !(in->contact_k[c] > 0.0f) ||
                    !(in->contact_area[c] > 0.0f) || !std::isfinite(in->contact_temp[c]))
                    return tfail(TG_ERR_INVALID_ARG, "contacts need cells in range, k > 0, area > 0, finite temperature");
            const size_t need = 4 * (G1 + 4 * C) + 64;
            if (need > t->scratch_cap) {
                TCK(cudaStreamSynchronize(st));
                if (t->scratch) cudaFree(t->scratch);
                t->scratch = nullptr;
                t->scratch_cap = 0;
                TCK(cudaMalloc(&t->scratch, need));
                t->scratch_cap = need;
            }
            char* p = (char*)t->scratch;
            auto put = [&](const void* src, size_t bytes) {
                void* dst = p;
                cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
                p += (bytes + 15) & ~(size_t)15;
                return dst;
            };
            a.c_off = (const int32_t*)put(in->contact_offsets, 4 * G1);
            a.c_cell = (const int32_t*)put(in->contact_cell, 4 * C);
            a.c_temp = (const float*)put(in->contact_temp, 4 * C);
            a.c_k = (const float*)put(in->contact_k, 4 * C);
            a.c_area = (const float*)put(in->contact_area, 4 * C);
            TCK(cudaStreamSynchronize(st));  // the host arrays may die at return
        }
    }
    temp_step_kernel<<<t->G, kTempThreads, t->smem, st>>>(a);
    TCK(cudaGetLastError());
    return TG_OK;
}

tg_status tg_temp_read(tg_temp* t, int32_t measured, float* dst, size_t dst_bytes, tg_stream stream) {
    if (!t || !dst) return tfail(TG_ERR_INVALID_ARG, "grid and dst are required");
    const size_t bytes = sizeof(float) * t->nx * t->ny * t->nz * t->G;
    if (dst_bytes != bytes) return tfail(TG_ERR_INVALID_ARG, "dst_bytes must be 4 * G * nx * ny * nz");
    TCK(cudaMemcpyAsync(dst, measured ? t->Tm : t->T, bytes, cudaMemcpyDefault, (cudaStream_t)stream));
    return TG_OK;
}

tg_status tg_temp_buffer(tg_temp* t, int32_t measured, float** ptr) {
    if (!t || !ptr) return tfail(TG_ERR_INVALID_ARG, "grid and ptr are required");
    *ptr = measured ? t->Tm : t->T;
    return TG_OK;
}

tg_status tg_contact_area(const float* points, const int32_t* n_points, const float* depth, int32_t n_pairs,
                          int32_t max_points, double d_w, float* area, tg_stream stream) {
    if (n_pairs < 0 || max_points < 1 || max_points > 16 || !std::isfinite(d_w))
        return tfail(TG_ERR_INVALID_ARG, "n_pairs >= 0, max_points in 1..16 and a finite d_w are required");
    if (n_pairs == 0) return TG_OK;
    if (!points || !n_points || !depth || !area || !t_is_dev(points) || !t_is_dev(n_points) || !t_is_dev(depth) ||
        !t_is_dev(area))
        return tfail(TG_ERR_INVALID_ARG, "points, n_points, depth and area must be device buffers");
    contact_area_kernel<<<(n_pairs + 127) / 128, 128, 0, (cudaStream_t)stream>>>(points, n_points, depth, n_pairs,
                                                                                max_points, (float)d_w, area);
    TCK(cudaGetLastError());
    return TG_OK;
}

const char* tg_temp_last_error(void) { return g_temp_error.c_str(); }

}  // extern "C"
