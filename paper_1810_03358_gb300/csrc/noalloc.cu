// Allocation-free variant of the non-bonded pair energy + gradient.
//
// Some callers cannot let a library allocate device memory: an application
// that runs inside another framework's memory pool with a hard cap, or a
// real-time loop that cannot afford cudaMalloc's implicit device
// synchronisation.  ffmin_pair_energy_grad_noalloc serves them: the caller
// passes device buffers for the inputs and outputs, and the only scratch it
// needs (partial row sums, block energies, a ticket counter) lives in the
// file-scope device array `g_noalloc_scratch` below, which every GPU that
// loads this library holds until the process exits.
//
// Computation: the same FP64 row sweep as the main pair kernel, over all
// i < j pairs of one system, Coulomb + Lennard-Jones, no bonded terms:
// rows of 128 i-atoms against 8 j-chunks, partial rows to the scratch, then
// one thread per atom sums its chunks in a fixed order and the last block
// sums the block energies and flags a non-finite energy or gradient (two
// coincident atoms), which the call reports after synchronising its stream.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "ffmin.h"

namespace {

constexpr int NA_TI = 128;      // i atoms per block (one per thread)
constexpr int NA_TJ = 128;      // j atoms staged per shared-memory tile
constexpr int NA_CHUNKS = 8;    // j chunks per row
constexpr int NA_MAX_ATOMS = 8192;
constexpr int NA_MAX_BLOCKS = (NA_MAX_ATOMS + NA_TI - 1) / NA_TI;
// doubles: partial rows [chunk][atom][4], block energies, one 8-byte word
// holding the last-block ticket and the non-finite flag (two uint32)
constexpr size_t NA_SCRATCH = (size_t)NA_CHUNKS * NA_MAX_ATOMS * 4 + NA_MAX_BLOCKS + 1;

__device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH];

constexpr int NA_MAX_DEVICES = 64;
// device address of the array per device ordinal, looked up once in the
// device's primary context (a cudaDeviceReset or another context would need
// a new lookup); the lock guards the first lookup against concurrent callers
double *g_scratch_ptr[NA_MAX_DEVICES];
std::mutex g_scratch_lock;

struct NaArgs {
    const double *x, *q, *sigma, *eps;
    int n;
    double sqrt_c;
    double *g, *e;
    double *part;      // [NA_CHUNKS][NA_MAX_ATOMS][4]
    double *eblock;    // [NA_MAX_BLOCKS]
    unsigned int *ticket;  // [0] last-block ticket, [1] non-finite flag
};

__device__ __forceinline__ void na_atom(const NaArgs &a, int j, double4_32a &p, double2 &c) {
    if (j < a.n) {
        const double s3 = a.sigma[j] * a.sigma[j] * a.sigma[j];
        const double w = sqrt(24.0 * a.eps[j]);
        p = make_double4_32a(a.x[3 * j], a.x[3 * j + 1], a.x[3 * j + 2], a.q[j] * a.sqrt_c);
        c = make_double2(w * s3, w * s3 * s3);
    } else {  // padding atom: far away, no charge, no Lennard-Jones
        p = make_double4_32a(1e6, 1e6, 1e6, 0.0);
        c = make_double2(0.0, 0.0);
    }
}

__global__ void __launch_bounds__(NA_TI) k_na_rows(NaArgs a) {
    __shared__ double4_32a sp[NA_TJ];
    __shared__ double2 sc[NA_TJ];
    const int i = blockIdx.x * NA_TI + threadIdx.x;
    double4_32a pi;
    double2 ci;
    na_atom(a, i, pi, ci);
    if (i >= a.n) pi = make_double4_32a(-1e6, -1e6, -1e6, 0.0);
    const int chunk = blockIdx.y;
    const int len = (a.n + NA_CHUNKS - 1) / NA_CHUNKS;
    const int j0 = chunk * len, j1 = min(a.n, j0 + len);
    double gx = 0.0, gy = 0.0, gz = 0.0, e = 0.0;
    for (int jt = j0; jt < j1; jt += NA_TJ) {
        const int jl = jt + threadIdx.x;
        double4_32a pj;
        double2 cj;
        na_atom(a, jl < j1 ? jl : a.n, pj, cj);
        sp[threadIdx.x] = pj;
        sc[threadIdx.x] = cj;
        __syncthreads();
        for (int k = 0; k < NA_TJ; k++) {
            if (jt + k == i) continue;
            const double dx = sp[k].x - pi.x, dy = sp[k].y - pi.y, dz = sp[k].z - pi.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ri = rsqrt(r2);
            const double ri2 = ri * ri, ri6 = ri2 * ri2 * ri2;
            const double ec = pi.w * sp[k].w * ri;
            const double c6 = ci.x * sc[k].x, c12 = ci.y * sc[k].y;
            const double t1 = c12 * ri6 - c6;
            e += ec + ri6 * t1 * (1.0 / 6.0);
            const double f = (ri6 * (c12 * ri6 + t1) + ec) * ri2;
            gx += f * dx;
            gy += f * dy;
            gz += f * dz;
        }
        __syncthreads();
    }
    if (i < a.n) {
        double *p = a.part + ((size_t)chunk * NA_MAX_ATOMS + i) * 4;
        p[0] = gx; p[1] = gy; p[2] = gz; p[3] = e;
    }
}

__global__ void __launch_bounds__(NA_TI) k_na_final(NaArgs a) {
    __shared__ double se[NA_TI];
    const int i = blockIdx.x * NA_TI + threadIdx.x;
    double e = 0.0;
    bool bad = false;
    if (i < a.n) {
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int ch = 0; ch < NA_CHUNKS; ch++) {
            const double *p = a.part + ((size_t)ch * NA_MAX_ATOMS + i) * 4;
            g0 += p[0]; g1 += p[1]; g2 += p[2]; e += p[3];
        }
        a.g[3 * i] = g0; a.g[3 * i + 1] = g1; a.g[3 * i + 2] = g2;
        e *= 0.5;  // each pair appears in two rows
        bad = !isfinite(g0) || !isfinite(g1) || !isfinite(g2);
    }
    se[threadIdx.x] = e;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.ticket + 1, 1u);
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < NA_TI; t++) s += se[t];
        a.eblock[blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(a.ticket, 1u);
        if (t == gridDim.x - 1) {  // last block: total in block order
            __threadfence();
            double tot = 0.0;
            for (int b = 0; b < (int)gridDim.x; b++) tot += __ldcg(&a.eblock[b]);
            *a.e = tot;
            if (!isfinite(tot)) atomicOr(a.ticket + 1, 1u);
            *a.ticket = 0u;
        }
    }
}

}  // namespace

extern "C" ffmin_status ffmin_pair_energy_grad_noalloc(const double *x_dev, const double *charge_dev,
                                                      const double *sigma_dev, const double *epsilon_dev,
                                                      int32_t n_atoms, double coulomb_c, double *g_dev,
                                                      double *e_dev, void *cuda_stream) {
    if (n_atoms < 1 || n_atoms > NA_MAX_ATOMS || !x_dev || !charge_dev || !sigma_dev || !epsilon_dev ||
        !g_dev || !e_dev)
        return FFMIN_ERR_INVALID_ARG;  // sizes beyond the fixed scratch are refused
    if (!(coulomb_c >= 0.0) || !std::isfinite(coulomb_c)) return FFMIN_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return FFMIN_ERR_CUDA;
    double *scr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_lock);
        if (!g_scratch_ptr[dev]) {  // first call on this device: look up the array's device address
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FFMIN_ERR_CUDA;
            g_scratch_ptr[dev] = (double *)p;
        }
        scr = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    NaArgs a;
    a.x = x_dev; a.q = charge_dev; a.sigma = sigma_dev; a.eps = epsilon_dev;
    a.n = n_atoms;
    a.sqrt_c = std::sqrt(coulomb_c == 0.0 ? 1389.38757 / 4.184 : coulomb_c);
    a.g = g_dev;
    a.e = e_dev;
    a.part = scr;
    a.eblock = scr + (size_t)NA_CHUNKS * NA_MAX_ATOMS * 4;
    a.ticket = (unsigned int *)(a.eblock + NA_MAX_BLOCKS);
    // the ticket and the flag must start at zero on every call (the array
    // keeps the last call's contents)
    if (cudaMemsetAsync(a.ticket, 0, sizeof(double), s) != cudaSuccess) return FFMIN_ERR_CUDA;
    const int blocks = (n_atoms + NA_TI - 1) / NA_TI;
    k_na_rows<<<dim3(blocks, NA_CHUNKS), NA_TI, 0, s>>>(a);
    k_na_final<<<blocks, NA_TI, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return FFMIN_ERR_CUDA;
    // the status needs the flag: read it back (pageable host word) and wait
    unsigned int flag = 0u;
    if (cudaMemcpyAsync(&flag, a.ticket + 1, sizeof(flag), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FFMIN_ERR_CUDA;
    return flag ? FFMIN_ERR_NONFINITE : FFMIN_OK;
}
