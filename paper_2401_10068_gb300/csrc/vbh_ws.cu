// vbh_ws.cu -- the learned warm start declared in include/vbh_ws.h: a set
// encoder trained on the GPU by hand-written kernels (a tiled GEMM for every
// contraction of the forward and backward passes, BF16 matrices with FP32
// accumulation, split-K partials summed in a fixed order so every result is
// run-to-run deterministic), Adam on FP32 master weights, the features of a
// data set and the starting point of a fit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "vbh.h"
#include "vbh_error.h"
#include "vbh_ws.h"

namespace {

#define WS_CK(call) VBH_CHECK_CUDA(call)

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// GELU(z) = z Phi(z), Phi(z) = erfc(-z / sqrt 2) / 2
__device__ __forceinline__ float gelu(float z) { return z * 0.5f * erfcf(-z * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * erfcf(-z * 0.70710678118654752f) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// C[z][m][n] = sum over k in split z of A(m, k) B(n, k), with
// A(m, k) = A[m sam + k sak] and B(n, k) = B[n sbn + k sbk]; 64 x 64 tiles of
// C per block, K in steps of 16 through shared memory, 4 x 4 outputs per
// thread.  Split z covers k in [z kchunk, (z + 1) kchunk).
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(int Md, int Nd, int Kd, int kchunk, const TA *__restrict__ A,
                                                   long long sam, long long sak, const TB *__restrict__ B,
                                                   long long sbn, long long sbk, float *__restrict__ C)
{
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(Kd, kbeg + kchunk);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
        for (int e = tid; e < GT * GK; e += 256) {
            // walk along the unit stride so that neighbouring threads load neighbouring words
            const int mm = (sak == 1) ? e / GK : e % GT, kk = (sak == 1) ? e % GK : e / GT;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < Md && k < kend) ? to_f(A[m * sam + k * sak]) : 0.0f;
            const int nn = (sbk == 1) ? e / GK : e % GT, kb = (sbk == 1) ? e % GK : e / GT;
            const int n = n0 + nn, kq = k0 + kb;
            Bs[kb][nn] = (n < Nd && kq < kend) ? to_f(B[n * sbn + kq * sbk]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                av[i] = As[kk][ty * 4 + i];
                bv[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *Cz = C + size_t(blockIdx.z) * size_t(Md) * size_t(Nd);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < Md && n < Nd) Cz[size_t(m) * Nd + n] = acc[i][j];
        }
}

// out[idx] = sum_z P[z][idx] (+ bias[idx % Nd]); optionally Z = that and A = GELU(that).
__global__ void epilogue_kernel(long long total, int Nd, int splits, const float *P, const float *bias, float *Z,
                                float *A)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += P[z * total + i];
        if (bias) s += bias[i % Nd];
        if (Z) Z[i] = s;
        if (A) A[i] = gelu(s);
    }
}

// Pool[b][h] = (1/n) sum_i A[(b n + i) H + h]
__global__ void pool_kernel(int B, int n, int H, const float *A, float *Pool)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * H) return;
    const int b = idx / H, h = idx % H;
    float s = 0.0f;
    for (int i = 0; i < n; ++i) s += A[(size_t(b) * n + i) * H + h];
    Pool[idx] = s / float(n);
}

// dOut = 2 (Out - T) / (B P); loss = sum (Out - T)^2 / (B P) in FP64 (one block, fixed order)
__global__ void loss_kernel(int BP, const float *Out, const float *T, float *dOut, double *loss)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < BP; i += blockDim.x) {
        const float r = Out[i] - T[i];
        dOut[i] = 2.0f * r / float(BP);
        s += double(r) * double(r);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < blockDim.x; ++i) t += red[i];
        *loss = t / double(BP);
    }
}

// dZ = dA * GELU'(Z), elementwise
__global__ void gelu_back_kernel(long long total, const float *dA, const float *Z, float *dZ)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        dZ[i] = dA[i] * gelu_grad(Z[i]);
}

// dZ2[(b n + i) H + h] = dPool[b][h] / n * GELU'(Z2[...]): the mean pool's backward
__global__ void pool_back_kernel(long long rows, int n, int H, const float *dPool, const float *Z2, float *dZ2)
{
    const long long total = rows * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / H;
        const int h = int(i % H), b = int(r / n);
        dZ2[i] = dPool[size_t(b) * H + h] / float(n) * gelu_grad(Z2[i]);
    }
}

// column sums of X (rows x cols) in row chunks: part[c][col] = sum over chunk c
__global__ void colsum_kernel(long long rows, int cols, int chunk, const float *X, float *part)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    const long long r0 = (long long)blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float s = 0.0f;
    for (long long r = r0; r < r1; ++r) s += X[r * cols + col];
    part[(size_t)blockIdx.y * cols + col] = s;
}

// Adam on the FP32 parameters, then their BF16 copy
__global__ void adam_kernel(size_t np, float *theta, const float *g, float *m, float *v, __nv_bfloat16 *w16, float lr,
                            float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        theta[i] = th;
        w16[i] = __float2bfloat16_rn(th);
    }
}

__global__ void to_bf16_kernel(size_t np, const float *theta, __nv_bfloat16 *w16)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x)
        w16[i] = __float2bfloat16_rn(theta[i]);
}

// x[j] = [D (M), y, y^2, y D (M)] of observation floor(j V / n)
__global__ void features_kernel(const float *r, const float *d, long long V, int S, int n, float *x)
{
    const int M = S - 1, F = 2 * M + 2;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const long long i = (long long)j * V / n;
        const float *di = d + i * S;
        const float dS = di[M];
        const float y = r[i] - dS;
        float *xj = x + (size_t)j * F;
        for (int k = 0; k < M; ++k) {
            const float D = di[k] - dS;
            xj[k] = D;
            xj[M + 2 + k] = y * D;
        }
        xj[M] = y;
        xj[M + 1] = y * y;
    }
}

unsigned grid_for(long long total, int threads, int cap = 4096)
{
    long long g = (total + threads - 1) / threads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return unsigned(g);
}

// splitmix64 of a counter: a uniform double in [0, 1)
double hash_uniform(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return double(z >> 11) * (1.0 / 9007199254740992.0);
}

template <typename T>
int grow(T **p, size_t *cap, size_t n)
{
    if (*cap >= n && *p) return VBH_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        return VBH_ENOMEM;
    }
    *cap = n;
    return VBH_OK;
}

} // namespace

struct vbh_ws {
    int device = 0;
    cudaStream_t stream = nullptr;
    int S = 0, M = 0, F = 0, P = 0, H = 0;
    size_t np = 0;
    size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, oW4 = 0, ob4 = 0;
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    __nv_bfloat16 *w16 = nullptr;
    std::vector<float> mean, std;
    int step = 0;
    // activations
    float *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *dZ2 = nullptr, *dA1 = nullptr;
    size_t cap_rows = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0;
    float *Pool = nullptr, *Z3 = nullptr, *A3 = nullptr, *Out = nullptr, *dOut = nullptr, *dZ3 = nullptr,
          *dPool = nullptr;
    size_t cb[7] = {0, 0, 0, 0, 0, 0, 0};
    float *part = nullptr;
    size_t cap_part = 0;
    float *scratch_x = nullptr, *scratch_out = nullptr;
    size_t cap_sx = 0, cap_so = 0;
    double *dloss = nullptr;
};

namespace {

struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev)
    {
        ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess;
        if (!ok) (void)cudaGetLastError();
    }
    ~Guard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename TA, typename TB>
int gemm(vbh_ws *m, int Md, int Nd, int Kd, int splits, const TA *A, long long sam, long long sak, const TB *B,
         long long sbn, long long sbk, float *C)
{
    if (Md == 0 || Nd == 0) return VBH_OK;
    const int kchunk = ((Kd + splits - 1) / splits + GK - 1) / GK * GK;
    const int nz = (Kd + kchunk - 1) / kchunk;
    dim3 grid((Nd + GT - 1) / GT, (Md + GT - 1) / GT, nz > 0 ? nz : 1);
    gemm_kernel<TA, TB><<<grid, 256, 0, m->stream>>>(Md, Nd, Kd, kchunk, A, sam, sak, B, sbn, sbk, C);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

int splits_used(int Kd, int splits)
{
    const int kchunk = ((Kd + splits - 1) / splits + GK - 1) / GK * GK;
    return (Kd + kchunk - 1) / kchunk;
}

int ensure_rows(vbh_ws *m, long long rows)
{
    const size_t n = size_t(rows) * m->H;
    int rc;
    if ((rc = grow(&m->Z1, &m->c1, n)) || (rc = grow(&m->A1, &m->c2, n)) || (rc = grow(&m->Z2, &m->c3, n)) ||
        (rc = grow(&m->A2, &m->c4, n)))
        return rc;
    return VBH_OK;
}

int ensure_sets(vbh_ws *m, int B)
{
    const size_t bh = size_t(B) * m->H, bp = size_t(B) * m->P;
    int rc;
    if ((rc = grow(&m->Pool, &m->cb[0], bh)) || (rc = grow(&m->Z3, &m->cb[1], bh)) || (rc = grow(&m->A3, &m->cb[2], bh)) ||
        (rc = grow(&m->Out, &m->cb[3], bp)) || (rc = grow(&m->dOut, &m->cb[4], bp)) ||
        (rc = grow(&m->dZ3, &m->cb[5], bh)) || (rc = grow(&m->dPool, &m->cb[6], bh)))
        return rc;
    return VBH_OK;
}

// Forward of B sets of n observations: raw outputs in m->Out.
int forward(vbh_ws *m, int B, int n, const float *x)
{
    const long long R = (long long)B * n;
    const int H = m->H, F = m->F, P = m->P;
    int rc;
    if ((rc = ensure_rows(m, R)) || (rc = ensure_sets(m, B))) return rc;
    const __nv_bfloat16 *W = m->w16;
    if ((rc = gemm(m, int(R), H, F, 1, x, F, 1, W + m->oW1, F, 1, m->Z1))) return rc;
    epilogue_kernel<<<grid_for(R * H, 256), 256, 0, m->stream>>>(R * H, H, 1, m->Z1, m->theta + m->ob1, m->Z1, m->A1);
    if ((rc = gemm(m, int(R), H, H, 1, m->A1, H, 1, W + m->oW2, H, 1, m->Z2))) return rc;
    epilogue_kernel<<<grid_for(R * H, 256), 256, 0, m->stream>>>(R * H, H, 1, m->Z2, m->theta + m->ob2, m->Z2, m->A2);
    pool_kernel<<<grid_for((long long)B * H, 256, 1 << 20), 256, 0, m->stream>>>(B, n, H, m->A2, m->Pool);
    if ((rc = gemm(m, B, H, H, 1, m->Pool, H, 1, W + m->oW3, H, 1, m->Z3))) return rc;
    epilogue_kernel<<<grid_for((long long)B * H, 256), 256, 0, m->stream>>>((long long)B * H, H, 1, m->Z3,
                                                                            m->theta + m->ob3, m->Z3, m->A3);
    if ((rc = gemm(m, B, P, H, 1, m->A3, H, 1, W + m->oW4, H, 1, m->Out))) return rc;
    epilogue_kernel<<<grid_for((long long)B * P, 256), 256, 0, m->stream>>>((long long)B * P, P, 1, m->Out,
                                                                            m->theta + m->ob4, m->Out, nullptr);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

// Weight gradient G (Nout x Kin) = sum over rows of dY[r][i] X[r][j], rows split in chunks; the
// partials are summed in order into grad + off.
int weight_grad(vbh_ws *m, long long rows, int Nout, int Kin, const float *dY, const float *X, size_t off)
{
    const int splits = rows > 4096 ? int((rows + 2047) / 2048) : 1;
    const int nz = splits_used(int(rows), splits);
    int rc;
    if ((rc = grow(&m->part, &m->cap_part, size_t(nz) * Nout * Kin))) return rc;
    if ((rc = gemm(m, Nout, Kin, int(rows), splits, dY, 1, Nout, X, 1, Kin, m->part))) return rc;
    epilogue_kernel<<<grid_for((long long)Nout * Kin, 256), 256, 0, m->stream>>>((long long)Nout * Kin, Kin, nz,
                                                                                 m->part, nullptr, m->grad + off,
                                                                                 nullptr);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

int bias_grad(vbh_ws *m, long long rows, int cols, const float *dZ, size_t off)
{
    const int chunk = 2048;
    const int nz = int((rows + chunk - 1) / chunk);
    int rc;
    if ((rc = grow(&m->part, &m->cap_part, size_t(nz) * cols))) return rc;
    dim3 grid((cols + 127) / 128, nz);
    colsum_kernel<<<grid, 128, 0, m->stream>>>(rows, cols, chunk, dZ, m->part);
    epilogue_kernel<<<grid_for(cols, 256), 256, 0, m->stream>>>(cols, cols, nz, m->part, nullptr, m->grad + off, nullptr);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

// Loss and gradient (in m->grad) of B sets against target.
int backward(vbh_ws *m, int B, int n, const float *x, const float *target, double *loss)
{
    const long long R = (long long)B * n;
    const int H = m->H, F = m->F, P = m->P;
    int rc;
    if ((rc = forward(m, B, n, x))) return rc;
    if ((rc = grow(&m->dZ2, &m->c5, size_t(R) * H)) || (rc = grow(&m->dA1, &m->c6, size_t(R) * H))) return rc;
    loss_kernel<<<1, 256, 0, m->stream>>>(B * P, m->Out, target, m->dOut, m->dloss);
    const __nv_bfloat16 *W = m->w16;
    // head
    if ((rc = weight_grad(m, B, P, H, m->dOut, m->A3, m->oW4)) || (rc = bias_grad(m, B, P, m->dOut, m->ob4))) return rc;
    if ((rc = gemm(m, B, H, P, 1, m->dOut, P, 1, W + m->oW4, 1, H, m->dZ3))) return rc;          // dA3 = dOut W4
    gelu_back_kernel<<<grid_for((long long)B * H, 256), 256, 0, m->stream>>>((long long)B * H, m->dZ3, m->Z3, m->dZ3);
    if ((rc = weight_grad(m, B, H, H, m->dZ3, m->Pool, m->oW3)) || (rc = bias_grad(m, B, H, m->dZ3, m->ob3))) return rc;
    if ((rc = gemm(m, B, H, H, 1, m->dZ3, H, 1, W + m->oW3, 1, H, m->dPool))) return rc;         // dPool = dZ3 W3
    // per observation
    pool_back_kernel<<<grid_for(R * H, 256), 256, 0, m->stream>>>(R, n, H, m->dPool, m->Z2, m->dZ2);
    if ((rc = weight_grad(m, R, H, H, m->dZ2, m->A1, m->oW2)) || (rc = bias_grad(m, R, H, m->dZ2, m->ob2))) return rc;
    if ((rc = gemm(m, int(R), H, H, 1, m->dZ2, H, 1, W + m->oW2, 1, H, m->dA1))) return rc;      // dA1 = dZ2 W2
    gelu_back_kernel<<<grid_for(R * H, 256), 256, 0, m->stream>>>(R * H, m->dA1, m->Z1, m->dA1);  // -> dZ1
    if ((rc = weight_grad(m, R, H, F, m->dA1, x, m->oW1)) || (rc = bias_grad(m, R, H, m->dA1, m->ob1))) return rc;
    WS_CK(cudaGetLastError());
    if (loss) {
        WS_CK(cudaMemcpyAsync(loss, m->dloss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    }
    return VBH_OK;
}

// B n <= 2^20 rows (the GEMM grid's y extent and the activation memory stay bounded)
bool shapes_ok(const vbh_ws *m, int B, int n) { return m && B >= 1 && n >= 1 && (long long)B * n <= (1LL << 20); }

} // namespace

extern "C" {

int vbh_ws_create(vbh_ws **mp, int S, int hidden, uint64_t seed, int device, void *stream)
{
    if (!mp) return VBH_EINVAL;
    *mp = nullptr;
    if (S < 2 || S > 11 || hidden < 64 || hidden > 1024 || hidden % 64) return VBH_EINVAL;
    Guard g(device);
    if (!g.ok) return VBH_EINVAL;
    vbh_ws *m = new (std::nothrow) vbh_ws();
    if (!m) return VBH_ENOMEM;
    m->device = device;
    m->stream = static_cast<cudaStream_t>(stream);
    m->S = S;
    m->M = S - 1;
    m->F = 2 * m->M + 2;
    m->P = m->M + 1 + m->M * (m->M + 1) / 2;
    m->H = hidden;
    const size_t H = hidden, F = m->F, P = m->P;
    m->oW1 = 0;
    m->ob1 = m->oW1 + H * F;
    m->oW2 = m->ob1 + H;
    m->ob2 = m->oW2 + H * H;
    m->oW3 = m->ob2 + H;
    m->ob3 = m->oW3 + H * H;
    m->oW4 = m->ob3 + H;
    m->ob4 = m->oW4 + P * H;
    m->np = m->ob4 + P;
    m->mean.assign(P, 0.0f);
    m->std.assign(P, 1.0f);
    std::vector<float> init(m->np, 0.0f);
    struct Blk { size_t off, rows, cols; } blks[] = {{m->oW1, H, F}, {m->oW2, H, H}, {m->oW3, H, H}, {m->oW4, P, H}};
    for (const Blk &b : blks) {
        const double a = std::sqrt(6.0 / double(b.rows + b.cols));
        for (size_t i = 0; i < b.rows * b.cols; ++i) init[b.off + i] = float((2.0 * hash_uniform(seed, b.off + i) - 1.0) * a);
    }
    int rc = VBH_OK;
    size_t c = 0;
    if ((rc = grow(&m->theta, &c, m->np)) || (c = 0, rc = grow(&m->grad, &c, m->np)) ||
        (c = 0, rc = grow(&m->am, &c, m->np)) || (c = 0, rc = grow(&m->av, &c, m->np)) ||
        (c = 0, rc = grow(&m->w16, &c, m->np)) || (c = 0, rc = grow(&m->dloss, &c, size_t(1)))) {
        vbh_ws_destroy(m);
        return rc;
    }
    if ((rc = vbh_ws_set_params(m, init.data(), init.size()))) {
        vbh_ws_destroy(m);
        return rc;
    }
    *mp = m;
    return VBH_OK;
}

void vbh_ws_destroy(vbh_ws *m)
{
    if (!m) return;
    Guard g(m->device);
    cudaStreamSynchronize(m->stream);
    float *bufs[] = {m->theta, m->grad, m->am, m->av, m->Z1, m->A1, m->Z2, m->A2, m->dZ2, m->dA1, m->Pool, m->Z3,
                     m->A3, m->Out, m->dOut, m->dZ3, m->dPool, m->part, m->scratch_x, m->scratch_out};
    for (float *p : bufs) cudaFree(p);
    cudaFree(m->w16);
    cudaFree(m->dloss);
    (void)cudaGetLastError();
    delete m;
}

int vbh_ws_sizes(const vbh_ws *m, int *F, int *P, size_t *nparams)
{
    if (!m) return VBH_EINVAL;
    if (F) *F = m->F;
    if (P) *P = m->P;
    if (nparams) *nparams = m->np;
    return VBH_OK;
}

int vbh_ws_get_params(vbh_ws *m, float *host, size_t n)
{
    if (!m || !host || n != m->np) return VBH_EINVAL;
    Guard g(m->device);
    WS_CK(cudaMemcpyAsync(host, m->theta, n * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
    return VBH_OK;
}

int vbh_ws_set_params(vbh_ws *m, const float *host, size_t n)
{
    if (!m || !host || n != m->np) return VBH_EINVAL;
    Guard g(m->device);
    WS_CK(cudaMemcpyAsync(m->theta, host, n * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    WS_CK(cudaMemsetAsync(m->am, 0, n * sizeof(float), m->stream));
    WS_CK(cudaMemsetAsync(m->av, 0, n * sizeof(float), m->stream));
    to_bf16_kernel<<<grid_for((long long)n, 256), 256, 0, m->stream>>>(n, m->theta, m->w16);
    WS_CK(cudaGetLastError());
    WS_CK(cudaStreamSynchronize(m->stream));
    m->step = 0;
    return VBH_OK;
}

int vbh_ws_set_norm(vbh_ws *m, const float *mean, const float *std)
{
    if (!m || !mean || !std) return VBH_EINVAL;
    for (int i = 0; i < m->P; ++i)
        if (!(std[i] > 0.0f) || !std::isfinite(mean[i])) return VBH_EINVAL;
    m->mean.assign(mean, mean + m->P);
    m->std.assign(std, std + m->P);
    return VBH_OK;
}

int vbh_ws_features(vbh_ws *m, const float *r, const float *d, int64_t V, int n, float *x)
{
    if (!m || !r || !d || !x || V < 1 || n < 1 || n > (1 << 20)) return VBH_EINVAL;
    Guard g(m->device);
    features_kernel<<<grid_for(n, 256), 256, 0, m->stream>>>(r, d, V, m->S, n, x);
    WS_CK(cudaGetLastError());
    WS_CK(cudaStreamSynchronize(m->stream));
    return VBH_OK;
}

int vbh_ws_forward(vbh_ws *m, int B, int n, const float *x, float *out)
{
    if (!shapes_ok(m, B, n) || !x || !out) return VBH_EINVAL;
    Guard g(m->device);
    int rc = forward(m, B, n, x);
    if (rc) return rc;
    WS_CK(cudaMemcpyAsync(out, m->Out, sizeof(float) * B * m->P, cudaMemcpyDeviceToDevice, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
    return VBH_OK;
}

int vbh_ws_loss_grad(vbh_ws *m, int B, int n, const float *x, const float *target, double *loss, float *grad)
{
    if (!shapes_ok(m, B, n) || !x || !target) return VBH_EINVAL;
    Guard g(m->device);
    int rc = backward(m, B, n, x, target, loss);
    if (rc) return rc;
    if (grad) WS_CK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
    return VBH_OK;
}

int vbh_ws_train_step(vbh_ws *m, int B, int n, const float *x, const float *target, float lr, double *loss)
{
    if (!shapes_ok(m, B, n) || !x || !target || !(lr > 0.0f)) return VBH_EINVAL;
    Guard g(m->device);
    int rc = backward(m, B, n, x, target, loss);
    if (rc) return rc;
    m->step += 1;
    const float c1 = float(1.0 - std::pow(0.9, m->step)), c2 = float(1.0 - std::pow(0.999, m->step));
    adam_kernel<<<grid_for((long long)m->np, 256), 256, 0, m->stream>>>(m->np, m->theta, m->grad, m->am, m->av, m->w16,
                                                                       lr, c1, c2);
    WS_CK(cudaGetLastError());
    WS_CK(cudaStreamSynchronize(m->stream));
    return VBH_OK;
}

int vbh_ws_predict(vbh_ws *m, const float *r, const float *d, int64_t V, const vbh_prior *p, int n, vbh_result *init)
{
    if (!m || !r || !d || !p || !init || V < 1 || n < 1 || n > (1 << 20) || p->S != m->S) return VBH_EINVAL;
    Guard g(m->device);
    int rc;
    if ((rc = grow(&m->scratch_x, &m->cap_sx, size_t(n) * m->F))) return rc;
    features_kernel<<<grid_for(n, 256), 256, 0, m->stream>>>(r, d, V, m->S, n, m->scratch_x);
    WS_CK(cudaGetLastError());
    if ((rc = forward(m, 1, n, m->scratch_x))) return rc;
    std::vector<float> out(m->P);
    WS_CK(cudaMemcpyAsync(out.data(), m->Out, sizeof(float) * m->P, cudaMemcpyDeviceToHost, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
    const int M = m->M;
    std::vector<double> t(m->P);
    for (int i = 0; i < m->P; ++i) t[i] = double(out[i]) * m->std[i] + m->mean[i];
    std::memset(init, 0, sizeof(*init));
    init->S = m->S;
    double sum = 0.0;
    for (int j = 0; j < M; ++j) {
        init->kappa[j] = t[j];
        init->weights[j] = t[j];
        sum += t[j];
    }
    init->weights[M] = 1.0 - sum;
    const double erho = std::exp(t[M]);
    std::vector<double> L(size_t(M) * M, 0.0);
    int o = M + 1;
    for (int j = 0; j < M; ++j)
        for (int k = 0; k <= j; ++k, ++o) L[size_t(j) * M + k] = (k == j) ? std::exp(t[o]) : t[o];
    const double Vd = double(V);
    init->nu = p->n0 + Vd;
    init->lambda = p->q0 + Vd;
    init->a_rho = p->a0 + 0.5 * Vd;
    init->b_rho = init->a_rho / erho;
    init->rho_mean = erho;
    init->rho_mode = (init->a_rho - 1.0) / init->b_rho;
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < M; ++k) {
            double s = 0.0;
            for (int q = 0; q <= (j < k ? j : k); ++q) s += L[size_t(j) * M + q] * L[size_t(k) * M + q];
            init->W_inv[j * M + k] = init->nu * s;                   // W^{-1} = nu Sigma0 (Eq. 28)
        }
    bool finite = std::isfinite(erho) && erho > 0.0;
    for (int i = 0; i < M * M; ++i) finite = finite && std::isfinite(init->W_inv[i]);
    return finite ? VBH_OK : VBH_ENONFINITE;
}

} // extern "C"
