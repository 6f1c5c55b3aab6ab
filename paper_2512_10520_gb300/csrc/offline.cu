// offline.cu -- the offline phase (Sec. Building histograms, Appendix A) on the
// GPU: histograms H[M][i] from a parametric physics sampler (a stand-in for
// the paper's Geant4 runs), the pilot estimator of Appendix A, and the
// bounded-variation momentum-bin edges built from it.
//
// Sampler, per sample s of stream h (h = material * n_pbin + bin for the
// histograms, the probe index for the pilot): eight uniforms
// u_j = (w >> 8 + 1/2) 2^-24 from Philox4x32-10 with key = seed and counters
// (s, h, 0x0FF1, 0) and (s, h, 0x0FF1, 1); u0 picks p in the bin; a Moyal
// ionisation loss xi (-ln z^2) + dmp (PDG thin-absorber xi and most probable
// loss with the density effect, z = sqrt(-2 ln u1) cos(2 pi u2)), floored at 0;
// with probability b rho x / <v> (u3) a radiative loss v ~ v^-2 on [1e-3, 1)
// (u4) added to f = dE / p; theta = theta0 sqrt(-2 ln u7), or 2 theta0 /
// sqrt(u6) when u5 < 0.01, theta0 the Highland width.  The arithmetic is FP64:
// the phase runs once per histogram set, and FP64 keeps every cell decision
// equal to the definition's.
#include <algorithm>
#include <cmath>
#include <vector>

#include "step.cuh"

namespace mt {
namespace {

constexpr double kK = 0.307075;        // MeV cm^2 / g
constexpr double kMe = 0.51099895;     // MeV
constexpr double kMmu = 105.6583755;   // MeV

struct Mat {
    double rho, za, I, X0, b;
};

__device__ __forceinline__ double u_open(uint32_t w) { return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }

__device__ __forceinline__ void uniforms8(uint32_t key0, uint32_t key1, uint32_t s, uint32_t h, double u[8])
{
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const uint4 w = philox4x32_10(make_uint4(s, h, 0x0FF1u, (uint32_t)half), key0, key1);
        u[4 * half + 0] = u_open(w.x);
        u[4 * half + 1] = u_open(w.y);
        u[4 * half + 2] = u_open(w.z);
        u[4 * half + 3] = u_open(w.w);
    }
}

__host__ __device__ inline double highland(double p_gev, double x_cm, double X0)
{
    const double pm = p_gev * 1e3;
    const double beta = pm / sqrt(pm * pm + kMmu * kMmu);
    const double t = x_cm / X0;
    return 13.6 / (beta * pm) * sqrt(t) * (1.0 + 0.038 * log(t));
}

// f = dp/p and theta of one sample at momentum p (GeV) through x_cm of m.
__device__ void physics_sample(const Mat &m, double p, double x_cm, const double u[8], double &f, double &theta)
{
    const double pm = p * 1e3;
    const double E = sqrt(pm * pm + kMmu * kMmu);
    const double beta2 = (pm / E) * (pm / E);
    const double bg = pm / kMmu;
    const double xi = 0.5 * kK * m.za * m.rho * x_cm / beta2;
    const double hw = 28.816e-6 * sqrt(m.rho * m.za);
    const double delta = fmax(0.0, 2.0 * log(bg) + 2.0 * log(hw / m.I) - 1.0);
    const double dmp = xi * (log(2.0 * kMe * bg * bg / m.I) + log(xi / m.I) + 0.2 - beta2 - delta);
    const double z = sqrt(-2.0 * log(u[1])) * cos(6.283185307179586476925286766559 * u[2]);
    const double z2 = fmax(z * z, 1e-300);
    double fl = fmax(dmp + xi * (-log(z2)), 0.0) / pm;
    const double v0 = 1e-3;
    const double mean_v = log(1.0 / v0) / (1.0 / v0 - 1.0);
    const double p_rad = fmin(1.0, m.b * m.rho * x_cm / mean_v);
    if (u[3] < p_rad) fl += 1.0 / (1.0 / v0 - u[4] * (1.0 / v0 - 1.0));
    const double th0 = highland(p, x_cm, m.X0);
    theta = u[5] < 0.01 ? 2.0 * th0 / sqrt(u[6]) : th0 * sqrt(-2.0 * log(u[7]));
    f = fl;
}

// Histogram h = blockIdx.y: blocks x = 0..gridDim.x-1 take samples
// s = x, x + gridDim.x, ... (by thread), count into a shared-memory histogram
// and add it to the global counts.
__global__ void __launch_bounds__(256) build_hist_kernel(const Mat *mats, int n_pbin, const double *edges,
                                                         int nf, int ntheta, double f_max, double x_cm,
                                                         int64_t n_samples, uint32_t key0, uint32_t key1,
                                                         const double *theta_max, unsigned int *counts)
{
    extern __shared__ unsigned int sh[];
    const int ncell = nf * ntheta;
    const int h = blockIdx.y;
    const int m = h / n_pbin, i = h % n_pbin;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) sh[c] = 0u;
    __syncthreads();
    const Mat mat = mats[m];
    const double pa = edges[i], pb = edges[i + 1], tm = theta_max[h];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_samples; s += stride) {
        double u[8], f, th;
        uniforms8(key0, key1, (uint32_t)s, (uint32_t)h, u);
        const double p = pa + u[0] * (pb - pa);
        physics_sample(mat, p, x_cm, u, f, th);
        double a = floor(f / f_max * nf), b = floor(th / tm * ntheta);
        a = (a >= 0.0) ? fmin(a, (double)(nf - 1)) : 0.0;
        b = (b >= 0.0) ? fmin(b, (double)(ntheta - 1)) : 0.0;
        atomicAdd(&sh[(int)a * ntheta + (int)b], 1u);
    }
    __syncthreads();
    unsigned int *out = counts + (int64_t)h * ncell;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x)
        if (sh[c]) atomicAdd(out + c, sh[c]);
}

__global__ void counts_to_double(const unsigned int *c, double *w, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        w[k] = (double)c[k];
}

// Pilot estimator: block (x, probe) sums log(-dPz/P) over its samples; the
// block sums are added in double.
__global__ void __launch_bounds__(256) pilot_kernel(Mat mat, const double *probes, int64_t K, double x_cm,
                                                    uint32_t key0, uint32_t key1, double *sums)
{
    __shared__ double part[8];
    const int j = blockIdx.y;
    const double p = probes[j];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < K; s += stride) {
        double u[8], f, th;
        uniforms8(key0, key1, (uint32_t)s, (uint32_t)j, u);
        physics_sample(mat, p, x_cm, u, f, th);
        f = fmin(f, 1.0);
        const double shh = sin(0.5 * th);
        acc += log(f + (1.0 - f) * 2.0 * shh * shh);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(sums + j, t);
    }
}

mt_status check_mat(const mt_material &m)
{
    if (!(m.rho > 0.0) || !(m.z_over_a > 0.0) || !(m.I_mev > 0.0) || !(m.X0_cm > 0.0) || !(m.b_rad >= 0.0) ||
        !std::isfinite(m.rho) || !std::isfinite(m.z_over_a) || !std::isfinite(m.I_mev) || !std::isfinite(m.X0_cm) ||
        !std::isfinite(m.b_rad)) {
        set_error("material: rho, Z/A, I and X0 must be positive and finite, b >= 0");
        return MT_ERR_INVALID_ARG;
    }
    return MT_OK;
}

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" {

mt_status mt_build_histograms(const mt_material *mats, int32_t n_mat, int32_t n_pbin, const double *edges, int32_t nf,
                              int32_t ntheta, double f_max, double step_len, int64_t n_samples, uint64_t seed,
                              double *weights, double *theta_max, void *stream)
{
    if (!mats || !edges || !weights || !theta_max || n_mat < 1 || n_mat > MT_MAX_MATERIALS || n_pbin < 1 ||
        n_pbin > MT_MAX_PBINS || nf < 1 || ntheta < 1 || (int64_t)nf * ntheta > MT_MAX_CELLS ||
        (int64_t)nf * ntheta < 2 || !(f_max > 0.0) || !(step_len > 0.0) || n_samples < 1 ||
        n_samples > 0xFFFFFFFFll) {
        set_error("build_histograms: bad arguments (null pointers, sizes out of range, f_max / step_len <= 0)");
        return MT_ERR_INVALID_ARG;
    }
    for (int m = 0; m < n_mat; ++m)
        if (check_mat(mats[m]) != MT_OK) return MT_ERR_INVALID_ARG;
    for (int i = 0; i < n_pbin; ++i)
        if (!(edges[i] > 0.0) || !(edges[i + 1] > edges[i]) || !std::isfinite(edges[i + 1])) {
            set_error("build_histograms: edges must be positive and increasing");
            return MT_ERR_INVALID_ARG;
        }
    const double x_cm = step_len * 100.0;
    const int64_t nh = (int64_t)n_mat * n_pbin, ncell = (int64_t)nf * ntheta;
    std::vector<Mat> hm(n_mat);
    for (int m = 0; m < n_mat; ++m)
        hm[m] = Mat{mats[m].rho, mats[m].z_over_a, mats[m].I_mev, mats[m].X0_cm, mats[m].b_rad};
    for (int64_t h = 0; h < nh; ++h) theta_max[h] = 5.0 * highland(edges[h % n_pbin], x_cm, hm[h / n_pbin].X0);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t b_mats = sizeof(Mat) * n_mat, b_edges = sizeof(double) * (n_pbin + 1), b_tm = sizeof(double) * nh;
    const size_t b_cnt = sizeof(unsigned int) * nh * ncell;
    char *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), b_mats + b_edges + b_tm + b_cnt + 1024, st);
    if (e != cudaSuccess) return cuda_fail(e, "build_histograms scratch");
    Mat *d_mats = reinterpret_cast<Mat *>(scratch);
    double *d_edges = reinterpret_cast<double *>(scratch + ((b_mats + 255) & ~(size_t)255));
    double *d_tm = reinterpret_cast<double *>((char *)d_edges + ((b_edges + 255) & ~(size_t)255));
    unsigned int *d_cnt = reinterpret_cast<unsigned int *>((char *)d_tm + ((b_tm + 255) & ~(size_t)255));
    e = cudaMemcpyAsync(d_mats, hm.data(), b_mats, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_edges, edges, b_edges, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tm, theta_max, b_tm, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, b_cnt, st);
    const size_t smem = sizeof(unsigned int) * ncell;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(build_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        // enough blocks per histogram to fill the GPU, each taking >= 4096 samples
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t bx = std::max<int64_t>(1, (int64_t)sms * 4 / nh);
        bx = std::min<int64_t>(bx, std::max<int64_t>(1, n_samples / 4096));
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        build_hist_kernel<<<dim3((unsigned)bx, (unsigned)nh), 256, smem, st>>>(
            d_mats, n_pbin, d_edges, nf, ntheta, f_max, x_cm, n_samples, k0, k1, d_tm, d_cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        counts_to_double<<<1024, 256, 0, st>>>(d_cnt, weights, nh * ncell);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = f;
    if (e != cudaSuccess) return cuda_fail(e, "build_histograms");
    return MT_OK;
}

mt_status mt_pilot_phi(const mt_material *mat, const double *probes, int32_t n_probe, int64_t K, double step_len,
                       uint64_t seed, double *phi, void *stream)
{
    if (!mat || !probes || !phi || n_probe < 1 || n_probe > 65535 || K < 1 || K > 0xFFFFFFFFll ||
        !(step_len > 0.0)) {
        set_error("pilot_phi: bad arguments");
        return MT_ERR_INVALID_ARG;
    }
    if (check_mat(*mat) != MT_OK) return MT_ERR_INVALID_ARG;
    for (int j = 0; j < n_probe; ++j)
        if (!(probes[j] > 0.0) || !std::isfinite(probes[j])) {
            set_error("pilot_phi: probe momenta must be positive and finite");
            return MT_ERR_INVALID_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    char *scratch = nullptr;
    const size_t b = sizeof(double) * n_probe;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), 2 * ((b + 255) & ~(size_t)255), st);
    if (e != cudaSuccess) return cuda_fail(e, "pilot scratch");
    double *d_probes = reinterpret_cast<double *>(scratch);
    double *d_sums = reinterpret_cast<double *>(scratch + ((b + 255) & ~(size_t)255));
    e = cudaMemcpyAsync(d_probes, probes, b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sums, 0, b, st);
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int64_t bx = std::max<int64_t>(1, (int64_t)sms * 8 / n_probe);
        bx = std::min<int64_t>(bx, std::max<int64_t>(1, K / 1024));
        const Mat m{mat->rho, mat->z_over_a, mat->I_mev, mat->X0_cm, mat->b_rad};
        pilot_kernel<<<dim3((unsigned)bx, (unsigned)n_probe), 256, 0, st>>>(
            m, d_probes, K, step_len * 100.0, (uint32_t)seed, (uint32_t)(seed >> 32), d_sums);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi, d_sums, b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const cudaError_t f = cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = f;
    if (e != cudaSuccess) return cuda_fail(e, "pilot_phi");
    for (int j = 0; j < n_probe; ++j) phi[j] /= (double)K;
    return MT_OK;
}

int32_t mt_bv_edges(const double *probes, const double *phi, int32_t n_probe, double eps, double *edges,
                    int32_t max_edges)
{
    if (!probes || !phi || !edges || n_probe < 2 || max_edges < 2 || !(eps >= 0.0)) {
        set_error("bv_edges: bad arguments");
        return -1;
    }
    for (int j = 0; j + 1 < n_probe; ++j)
        if (!(probes[j + 1] > probes[j])) {
            set_error("bv_edges: probes must increase");
            return -1;
        }
    int32_t n = 0, i = 0;
    edges[n++] = probes[0];
    while (i < n_probe - 1) {
        // largest j with max_{i < k <= j} |phi_k - phi_i| <= eps, at least i + 1
        int32_t j = i + 1;
        bool within = std::fabs(phi[j] - phi[i]) <= eps;
        while (within && j + 1 < n_probe && std::fabs(phi[j + 1] - phi[i]) <= eps) ++j;
        if (n >= max_edges) {
            set_error("bv_edges: more than %d edges", max_edges);
            return -1;
        }
        edges[n++] = probes[j];
        i = j;
    }
    return n;
}

}  // extern "C"
