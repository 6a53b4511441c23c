// vbh_ws.cu -- the learned warm start declared in include/vbh_ws.h: a set
// encoder over the observations of a data set, trained on the GPU.
//
// Per call a batch of data sets is laid out as rows of 128-row tiles (each
// data set starts on a tile boundary; its last tile is partly valid), the
// features of the pooled observations are formed on the device, and the two
// per-observation layers run as tcgen05 contractions (vbh_ws_tc.cuh) whose
// epilogues apply bias and GELU, write the BF16 activations in the operand
// layout of the next contraction, and sum the second layer's activations per
// tile for the mean pool.  The head works on one row per data set in FP32 on
// the CUDA cores.  The backward pass recomputes layer 2 with the gradient of
// the pool times GELU' in its epilogue (dZ2), contracts dZ2 with W2 into dZ1
// (epilogue: GELU' of the stored layer-1 pre-activations), and forms the
// weight gradients dZ2^T A1 and dZ1^T X as split-K contractions over the
// observations whose partials, like every other sum here, are added in a
// fixed order.
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
#include "vbh_ws_tc.cuh"

namespace {

using vbh::WsGemmArgs;
using vbh::tl_index;

constexpr int F = VBH_WS_F, P = VBH_WS_P, H = VBH_WS_HIDDEN, SMAXW = VBH_WS_SMAX;
constexpr int MMAXW = SMAXW - 1;
constexpr long long ROWS_MAX = 1LL << 26;
constexpr int SPLIT_ROWS = 8192;                 // observations per split of the weight-gradient contractions

#define WS_CK(call) VBH_CHECK_CUDA(call)

// ---------------------------------------------------------------------------
// Features (the slot layout of vbh_ws.h) of observation i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void feature_row(const float *__restrict__ r, const float *__restrict__ d, long long i,
                                            int S, float (&f)[F])
{
    const int M = S - 1;
    const float dS = d[i * S + M];
    const float y = r[i] - dS;
    const float y2 = y * y;
#pragma unroll
    for (int j = 0; j < F; ++j) f[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < MMAXW; ++j) {
        const float D = (j < M) ? d[i * S + j] - dS : 0.0f;
        f[j] = D;
        f[9 + j] = (j < M) ? 1.0f : 0.0f;
        f[20 + j] = y * D;
        f[29 + j] = y2 * D;
    }
    f[18] = y;
    f[19] = y2;
}

struct SetDesc {
    const float *r, *d;
    long long V, n, row0;       // observations, pooled observations, first row
    int S, tile0, ntiles, pad;
};

// One block per row tile, one thread per row: the features of the tile's rows
// in the K-major operand layout (and, for training, transposed: rows = the 64
// feature slots, cols = rows).
__global__ void features_kernel(const SetDesc *__restrict__ sets, const int *__restrict__ tile_set,
                                const int *__restrict__ tile_valid, long long Rpad, __nv_bfloat16 *__restrict__ X,
                                __nv_bfloat16 *__restrict__ XT)
{
    const int t = blockIdx.x, row = threadIdx.x;
    const SetDesc s = sets[tile_set[t]];
    const long long m = (long long)t * 128 + row;
    float f[F];
    if (row < tile_valid[t]) {
        const long long j = m - s.row0;
        const long long i = (s.n == s.V) ? j : (j * s.V) / s.n;
        feature_row(s.r, s.d, i, s.S, f);
    } else {
#pragma unroll
        for (int k = 0; k < F; ++k) f[k] = 0.0f;
    }
    float h[32];
#pragma unroll
    for (int a = 0; a < F / 32; ++a) {
#pragma unroll
        for (int k = 0; k < 32; ++k) h[k] = f[32 * a + k];
        vbh::store_row32_bf16(X, m, 32 * a, F, h);
    }
    if (XT) {
#pragma unroll 8
        for (int k = 0; k < F; ++k) XT[tl_index(k, m, Rpad, 64)] = __float2bfloat16_rn(f[k]);
    }
}

// The checking entry's features: FP32 row-major.
__global__ void features_f32_kernel(const float *r, const float *d, long long V, int S, long long n, float *x)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        float f[F];
        feature_row(r, d, (n == V) ? j : (j * V) / n, S, f);
#pragma unroll
        for (int k = 0; k < F; ++k) x[j * F + k] = f[k];
    }
}

// Pool[b][h] = (sum over the set's tiles of the tile sums) / n_b, tiles in order.
__global__ void pool_kernel(int B, const SetDesc *__restrict__ sets, const float *__restrict__ cs,
                            float *__restrict__ pool)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * H) return;
    const int b = idx / H, h = idx % H;
    const SetDesc s = sets[b];
    float acc = 0.0f;
    for (int t = s.tile0; t < s.tile0 + s.ntiles; ++t) acc += cs[(size_t)t * H + h];
    pool[idx] = acc / float(s.n);
}

// Head, one block of 256 threads per data set: Z3 = W3 p + b3, A3 = GELU(Z3),
// Out = W4 A3 + b4 (W3t, W4t: transposed FP32 copies, for coalesced reads).
__global__ void __launch_bounds__(256) head_forward_kernel(const float *__restrict__ pool,
                                                           const float *__restrict__ W3t,
                                                           const float *__restrict__ b3,
                                                           const float *__restrict__ W4t,
                                                           const float *__restrict__ b4, float *__restrict__ Z3,
                                                           float *__restrict__ A3, float *__restrict__ out)
{
    __shared__ float sp[H], sa[H];
    const int b = blockIdx.x, h = threadIdx.x;
    sp[h] = pool[(size_t)b * H + h];
    __syncthreads();
    float z = b3[h];
    for (int k = 0; k < H; ++k) z = fmaf(W3t[(size_t)k * H + h], sp[k], z);
    const float a = vbh::ws_gelu(z);
    Z3[(size_t)b * H + h] = z;
    A3[(size_t)b * H + h] = a;
    sa[h] = a;
    __syncthreads();
    if (h < P) {
        float o = b4[h];
        for (int k = 0; k < H; ++k) o = fmaf(W4t[(size_t)k * P + h], sa[k], o);
        out[(size_t)b * P + h] = o;
    }
}

// Loss sum w (out - t)^2 / B (FP64, one block, fixed order) and dOut = 2 w (out - t) / B.
__global__ void loss_kernel(int B, const float *out, const float *t, const float *w, float *dout, double *loss)
{
    __shared__ double red[256];
    const int n = B * P;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float e = out[i] - t[i];
        dout[i] = 2.0f * w[i] * e / float(B);
        s += double(w[i]) * double(e) * double(e);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < blockDim.x; ++i) a += red[i];
        *loss = a / double(B);
    }
}

// Head backward, one block per data set: dA3 = W4^T dOut, dZ3 = dA3 GELU'(Z3),
// dPool = W3^T dZ3.
__global__ void __launch_bounds__(256) head_backward_kernel(const float *__restrict__ dout,
                                                            const float *__restrict__ Z3,
                                                            const float *__restrict__ W4,
                                                            const float *__restrict__ W3, float *__restrict__ dZ3,
                                                            float *__restrict__ dpool)
{
    __shared__ float so[P], sz[H];
    const int b = blockIdx.x, h = threadIdx.x;
    if (h < P) so[h] = dout[(size_t)b * P + h];
    __syncthreads();
    float da = 0.0f;
    for (int p = 0; p < P; ++p) da = fmaf(W4[(size_t)p * H + h], so[p], da);
    const float dz = da * vbh::ws_gelu_grad(Z3[(size_t)b * H + h]);
    dZ3[(size_t)b * H + h] = dz;
    sz[h] = dz;
    __syncthreads();
    float dp = 0.0f;
    for (int k = 0; k < H; ++k) dp = fmaf(W3[(size_t)k * H + h], sz[k], dp);
    dpool[(size_t)b * H + h] = dp;
}

// G[i][j] = sum_b U[b][i] Wm[b][j] (b in order), gb[i] = sum_b U[b][i]: the head's
// weight and bias gradients over the data sets of the batch.
__global__ void outer_sum_kernel(int B, int NI, int NJ, const float *__restrict__ U, const float *__restrict__ Wm,
                                 float *__restrict__ G, float *__restrict__ gb)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NI * NJ) return;
    const int i = idx / NJ, j = idx % NJ;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s = fmaf(U[(size_t)b * NI + i], Wm[(size_t)b * NJ + j], s);
    G[idx] = s;
    if (j == 0) {
        float t = 0.0f;
        for (int b = 0; b < B; ++b) t += U[(size_t)b * NI + i];
        gb[i] = t;
    }
}

// out[i] = sum over k < nparts of part[k][i], in order (split-K partials, tile sums).
__global__ void sum_parts_kernel(long long n, int nparts, const float *__restrict__ part, float *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < nparts; ++k) s += part[(size_t)k * n + i];
        out[i] = s;
    }
}

// Adam on the FP32 parameters.
__global__ void adam_kernel(size_t np, float *theta, const float *g, float *m, float *v, float lr, float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

// The copies the kernels read, from the FP32 parameters: W1 (H x F) and W2 (H x H)
// in the B-operand layout (row blocks of 256), W2^T likewise, W3^T and W4^T in FP32.
__global__ void pack_kernel(const float *__restrict__ W1, const float *__restrict__ W2, const float *__restrict__ W3,
                            const float *__restrict__ W4, __nv_bfloat16 *__restrict__ W1b,
                            __nv_bfloat16 *__restrict__ W2b, __nv_bfloat16 *__restrict__ W2Tb,
                            float *__restrict__ W3t, float *__restrict__ W4t)
{
    const int tot = H * F + 2 * H * H + H * H + P * H;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        int k = e;
        if (k < H * F) {
            const int i = k / F, j = k % F;
            W1b[tl_index(i, j, F, 256)] = __float2bfloat16_rn(W1[k]);
            continue;
        }
        k -= H * F;
        if (k < H * H) {
            const int i = k / H, j = k % H;
            W2b[tl_index(i, j, H, 256)] = __float2bfloat16_rn(W2[k]);
            W2Tb[tl_index(j, i, H, 256)] = __float2bfloat16_rn(W2[k]);
            continue;
        }
        k -= H * H;
        if (k < H * H) {
            const int i = k / H, j = k % H;
            W3t[(size_t)j * H + i] = W3[k];
            continue;
        }
        k -= H * H;
        if (k < P * H) {
            const int i = k / H, j = k % H;
            W4t[(size_t)j * P + i] = W4[k];
        }
    }
}

unsigned grid_for(long long total, int threads, int cap = 8192)
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
    if (n == 0) return VBH_OK;
    if (cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        return VBH_ENOMEM;
    }
    *cap = n;
    return VBH_OK;
}

template <typename T>
struct Buf {
    T *p = nullptr;
    size_t cap = 0;
    int need(size_t n) { return grow(&p, &cap, n); }
    void release()
    {
        cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

} // namespace

struct vbh_ws {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 148;
    size_t np = 0;
    size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, oW4 = 0, ob4 = 0;
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr;
    float *W3t = nullptr, *W4t = nullptr;
    std::vector<float> mean, std;
    int step = 0;
    int *err = nullptr;
    double *dloss = nullptr;
    // batch plan
    Buf<SetDesc> sets;
    Buf<int> tile_set, tile_valid;
    Buf<float> inv_count;
    // per-row activations and their gradients
    Buf<__nv_bfloat16> X, XT, A1, A1T, dZ2, dZ2T, dZ1T;
    Buf<float> Z1, cs, csd2, csd1;
    // per-set values
    Buf<float> pool, Z3, A3, out, dout, dZ3, dpool, parts;
    long long rpad = 0;
    int ntiles = 0, nsets = 0;
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

template <int NT, int EPI>
int launch_gemm(vbh_ws *m, WsGemmArgs a, int splits)
{
    using C = vbh::WsGemmCfg<NT>;
    static bool attr = false;
    if (!attr) {
        WS_CK(cudaFuncSetAttribute(vbh::ws_gemm_kernel<NT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(C::SMEM_BYTES)));
        attr = true;
    }
    a.err = m->err;
    const long long items = (long long)(a.M / 128) * (a.N / NT) * splits;
    const unsigned grid = unsigned(items < m->nsm ? items : m->nsm);     // persistent: one block per SM
    vbh::ws_gemm_kernel<NT, EPI><<<grid, C::THREADS, C::SMEM_BYTES, m->stream>>>(a);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

// Lay out a batch: data sets on 128-row tile boundaries, the features of
// their pooled observations (and, for training, transposed).
int plan_batch(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V, const int *S,
               const int64_t *n, bool training)
{
    if (B < 1 || !r || !d || !V || !S) return VBH_EINVAL;
    std::vector<SetDesc> sd(B);
    std::vector<int> tset, tvalid;
    std::vector<float> invc(B);
    long long rows = 0;
    for (int b = 0; b < B; ++b) {
        if (!r[b] || !d[b] || V[b] < 1 || S[b] < 2 || S[b] > SMAXW) return VBH_EINVAL;
        if (n && n[b] > 0 && n[b] < V[b] && V[b] > (1LL << 36)) return VBH_EINVAL;   // j V fits in 64 bits
        if (reinterpret_cast<uintptr_t>(r[b]) % 16 || reinterpret_cast<uintptr_t>(d[b]) % 16) return VBH_EINVAL;
        const long long nb = (n && n[b] > 0 && n[b] < V[b]) ? n[b] : V[b];
        const int nt = int((nb + 127) / 128);
        sd[b] = SetDesc{r[b], d[b], V[b], nb, rows, S[b], int(tset.size()), nt, 0};
        for (int t = 0; t < nt; ++t) {
            tset.push_back(b);
            tvalid.push_back(int(std::min<long long>(128, nb - 128LL * t)));
        }
        invc[b] = float(1.0 / double(nb));
        rows += 128LL * nt;
        if (rows > ROWS_MAX) return VBH_EINVAL;
    }
    const int nt = int(tset.size());
    int rc;
    if ((rc = m->sets.need(B)) || (rc = m->tile_set.need(nt)) || (rc = m->tile_valid.need(nt)) ||
        (rc = m->inv_count.need(B)))
        return rc;
    WS_CK(cudaMemcpyAsync(m->sets.p, sd.data(), sizeof(SetDesc) * B, cudaMemcpyHostToDevice, m->stream));
    WS_CK(cudaMemcpyAsync(m->tile_set.p, tset.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, m->stream));
    WS_CK(cudaMemcpyAsync(m->tile_valid.p, tvalid.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, m->stream));
    WS_CK(cudaMemcpyAsync(m->inv_count.p, invc.data(), sizeof(float) * B, cudaMemcpyHostToDevice, m->stream));
    if ((rc = m->X.need(size_t(rows) * F))) return rc;
    if (training && (rc = m->XT.need(size_t(rows) * F))) return rc;
    features_kernel<<<nt, 128, 0, m->stream>>>(m->sets.p, m->tile_set.p, m->tile_valid.p, rows, m->X.p,
                                               training ? m->XT.p : nullptr);
    WS_CK(cudaGetLastError());
    // the host vectors above are read by the copies: wait before they go
    WS_CK(cudaStreamSynchronize(m->stream));
    m->rpad = rows;
    m->ntiles = nt;
    m->nsets = B;
    return VBH_OK;
}

// Forward of the planned batch: raw outputs in m->out.  training keeps Z1 and
// A1^T for the backward pass.
int forward(vbh_ws *m, bool training)
{
    const long long R = m->rpad;
    const int B = m->nsets, nt = m->ntiles;
    int rc;
    if ((rc = m->A1.need(size_t(R) * H)) || (rc = m->cs.need(size_t(nt) * H))) return rc;
    if (training && ((rc = m->Z1.need(size_t(R) * H)) || (rc = m->A1T.need(size_t(R) * H)))) return rc;
    if ((rc = m->pool.need(size_t(B) * H)) || (rc = m->Z3.need(size_t(B) * H)) || (rc = m->A3.need(size_t(B) * H)) ||
        (rc = m->out.need(size_t(B) * P)))
        return rc;
    WsGemmArgs a{};
    a.A = m->X.p;
    a.B = m->W1b;
    a.M = int(R);
    a.N = H;
    a.K = F;
    a.kchunk = F;
    a.bias = m->theta + m->ob1;
    a.Z = training ? m->Z1.p : nullptr;
    a.Aout = m->A1.p;
    a.ATout = training ? m->A1T.p : nullptr;
    a.rbt = 256;
    a.Mt = R;
    a.valid = m->tile_valid.p;
    if ((rc = launch_gemm<256, vbh::EPI_FWD>(m, a, 1))) return rc;
    WsGemmArgs b{};
    b.A = m->A1.p;
    b.B = m->W2b;
    b.M = int(R);
    b.N = H;
    b.K = H;
    b.kchunk = H;
    b.bias = m->theta + m->ob2;
    b.colsum = m->cs.p;
    b.valid = m->tile_valid.p;
    if ((rc = launch_gemm<256, vbh::EPI_FWD>(m, b, 1))) return rc;
    pool_kernel<<<grid_for((long long)B * H, 256), 256, 0, m->stream>>>(B, m->sets.p, m->cs.p, m->pool.p);
    head_forward_kernel<<<B, 256, 0, m->stream>>>(m->pool.p, m->W3t, m->theta + m->ob3, m->W4t, m->theta + m->ob4,
                                                  m->Z3.p, m->A3.p, m->out.p);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

// Loss and gradient (in m->grad) of the planned batch.
int backward(vbh_ws *m, const float *target, const float *weight, double *loss)
{
    const long long R = m->rpad;
    const int B = m->nsets, nt = m->ntiles;
    int rc;
    if ((rc = forward(m, true))) return rc;
    if ((rc = m->dout.need(size_t(B) * P)) || (rc = m->dZ3.need(size_t(B) * H)) || (rc = m->dpool.need(size_t(B) * H)))
        return rc;
    if ((rc = m->dZ2.need(size_t(R) * H)) || (rc = m->dZ2T.need(size_t(R) * H)) || (rc = m->dZ1T.need(size_t(R) * H)) ||
        (rc = m->csd2.need(size_t(nt) * H)) || (rc = m->csd1.need(size_t(nt) * H)))
        return rc;
    const int splits = int((R + SPLIT_ROWS - 1) / SPLIT_ROWS);
    if ((rc = m->parts.need(size_t(splits) * H * H))) return rc;
    loss_kernel<<<1, 256, 0, m->stream>>>(B, m->out.p, target, weight, m->dout.p, m->dloss);
    head_backward_kernel<<<B, 256, 0, m->stream>>>(m->dout.p, m->Z3.p, m->theta + m->oW4, m->theta + m->oW3, m->dZ3.p,
                                                   m->dpool.p);
    outer_sum_kernel<<<grid_for(P * H, 256), 256, 0, m->stream>>>(B, P, H, m->dout.p, m->A3.p, m->grad + m->oW4,
                                                                  m->grad + m->ob4);
    outer_sum_kernel<<<grid_for(H * H, 256), 256, 0, m->stream>>>(B, H, H, m->dZ3.p, m->pool.p, m->grad + m->oW3,
                                                                  m->grad + m->ob3);
    WS_CK(cudaGetLastError());
    // dZ2 = dPool / n * GELU'(Z2): layer 2 again, the derivative in the epilogue
    WsGemmArgs a{};
    a.A = m->A1.p;
    a.B = m->W2b;
    a.M = int(R);
    a.N = H;
    a.K = H;
    a.kchunk = H;
    a.bias = m->theta + m->ob2;
    a.Aout = m->dZ2.p;
    a.ATout = m->dZ2T.p;
    a.rbt = 128;
    a.Mt = R;
    a.colsum = m->csd2.p;
    a.valid = m->tile_valid.p;
    a.tile_set = m->tile_set.p;
    a.dpool = m->dpool.p;
    a.inv_count = m->inv_count.p;
    if ((rc = launch_gemm<256, vbh::EPI_DZ2>(m, a, 1))) return rc;
    // dZ1 = (dZ2 W2) GELU'(Z1)
    WsGemmArgs b{};
    b.A = m->dZ2.p;
    b.B = m->W2Tb;
    b.M = int(R);
    b.N = H;
    b.K = H;
    b.kchunk = H;
    b.Zin = m->Z1.p;
    b.ATout = m->dZ1T.p;
    b.rbt = 128;
    b.Mt = R;
    b.colsum = m->csd1.p;
    b.valid = m->tile_valid.p;
    if ((rc = launch_gemm<256, vbh::EPI_BWD>(m, b, 1))) return rc;
    // dW2 = dZ2^T A1 and dW1 = dZ1^T X over the rows, split-K, partials in order
    const int kchunk = SPLIT_ROWS;
    WsGemmArgs c{};
    c.A = m->dZ2T.p;
    c.B = m->A1T.p;
    c.M = H;
    c.N = H;
    c.K = int(R);
    c.kchunk = kchunk;
    c.out = m->parts.p;
    if ((rc = launch_gemm<256, vbh::EPI_PLAIN>(m, c, splits))) return rc;
    sum_parts_kernel<<<grid_for(H * H, 256), 256, 0, m->stream>>>(H * H, splits, m->parts.p, m->grad + m->oW2);
    WsGemmArgs e{};
    e.A = m->dZ1T.p;
    e.B = m->XT.p;
    e.M = H;
    e.N = F;
    e.K = int(R);
    e.kchunk = kchunk;
    e.out = m->parts.p;
    if ((rc = launch_gemm<64, vbh::EPI_PLAIN>(m, e, splits))) return rc;
    sum_parts_kernel<<<grid_for(H * F, 256), 256, 0, m->stream>>>(H * F, splits, m->parts.p, m->grad + m->oW1);
    sum_parts_kernel<<<grid_for(H, 256), 256, 0, m->stream>>>(H, nt, m->csd2.p, m->grad + m->ob2);
    sum_parts_kernel<<<grid_for(H, 256), 256, 0, m->stream>>>(H, nt, m->csd1.p, m->grad + m->ob1);
    WS_CK(cudaGetLastError());
    if (loss) WS_CK(cudaMemcpyAsync(loss, m->dloss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    return VBH_OK;
}

int check_err(vbh_ws *m)
{
    int e = 0;
    WS_CK(cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
    return e;
}

int pack(vbh_ws *m)
{
    pack_kernel<<<grid_for(H * F + 3 * H * H + P * H, 256), 256, 0, m->stream>>>(
        m->theta + m->oW1, m->theta + m->oW2, m->theta + m->oW3, m->theta + m->oW4, m->W1b, m->W2b, m->W2Tb, m->W3t,
        m->W4t);
    WS_CK(cudaGetLastError());
    return VBH_OK;
}

} // namespace

extern "C" {

int vbh_ws_create(vbh_ws **mp, uint64_t seed, int device, void *stream)
{
    if (!mp) return VBH_EINVAL;
    *mp = nullptr;
    Guard g(device);
    if (!g.ok) return VBH_EINVAL;
    vbh_ws *m = new (std::nothrow) vbh_ws();
    if (!m) return VBH_ENOMEM;
    if (cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || m->nsm < 1) {
        (void)cudaGetLastError();
        delete m;
        return VBH_ECUDA;
    }
    m->device = device;
    m->stream = static_cast<cudaStream_t>(stream);
    m->oW1 = 0;
    m->ob1 = m->oW1 + size_t(H) * F;
    m->oW2 = m->ob1 + H;
    m->ob2 = m->oW2 + size_t(H) * H;
    m->oW3 = m->ob2 + H;
    m->ob3 = m->oW3 + size_t(H) * H;
    m->oW4 = m->ob3 + H;
    m->ob4 = m->oW4 + size_t(P) * H;
    m->np = m->ob4 + P;
    m->mean.assign(size_t(SMAXW + 1) * P, 0.0f);
    m->std.assign(size_t(SMAXW + 1) * P, 1.0f);
    std::vector<float> init(m->np, 0.0f);
    struct Blk {
        size_t off, rows, cols;
    } blks[] = {{m->oW1, H, F}, {m->oW2, H, H}, {m->oW3, H, H}, {m->oW4, P, H}};
    for (const Blk &b : blks) {
        const double a = std::sqrt(6.0 / double(b.rows + b.cols));
        for (size_t i = 0; i < b.rows * b.cols; ++i)
            init[b.off + i] = float((2.0 * hash_uniform(seed, b.off + i) - 1.0) * a);
    }
    int rc = VBH_OK;
    size_t c = 0;
    if ((rc = grow(&m->theta, &c, m->np)) || (c = 0, rc = grow(&m->grad, &c, m->np)) ||
        (c = 0, rc = grow(&m->am, &c, m->np)) || (c = 0, rc = grow(&m->av, &c, m->np)) ||
        (c = 0, rc = grow(&m->W1b, &c, size_t(H) * F)) || (c = 0, rc = grow(&m->W2b, &c, size_t(H) * H)) ||
        (c = 0, rc = grow(&m->W2Tb, &c, size_t(H) * H)) || (c = 0, rc = grow(&m->W3t, &c, size_t(H) * H)) ||
        (c = 0, rc = grow(&m->W4t, &c, size_t(P) * H)) || (c = 0, rc = grow(&m->dloss, &c, size_t(1))) ||
        (c = 0, rc = grow(&m->err, &c, size_t(1)))) {
        vbh_ws_destroy(m);
        return rc;
    }
    if (cudaMemsetAsync(m->err, 0, sizeof(int), m->stream) != cudaSuccess ||
        (rc = vbh_ws_set_params(m, init.data(), init.size()))) {
        vbh_ws_destroy(m);
        return rc ? rc : VBH_ECUDA;
    }
    *mp = m;
    return VBH_OK;
}

void vbh_ws_destroy(vbh_ws *m)
{
    if (!m) return;
    Guard g(m->device);
    cudaStreamSynchronize(m->stream);
    float *fb[] = {m->theta, m->grad, m->am, m->av, m->W3t, m->W4t};
    for (float *p : fb) cudaFree(p);
    cudaFree(m->W1b);
    cudaFree(m->W2b);
    cudaFree(m->W2Tb);
    cudaFree(m->dloss);
    cudaFree(m->err);
    m->sets.release();
    m->tile_set.release();
    m->tile_valid.release();
    m->inv_count.release();
    m->X.release();
    m->XT.release();
    m->A1.release();
    m->A1T.release();
    m->dZ2.release();
    m->dZ2T.release();
    m->dZ1T.release();
    m->Z1.release();
    m->cs.release();
    m->csd2.release();
    m->csd1.release();
    m->pool.release();
    m->Z3.release();
    m->A3.release();
    m->out.release();
    m->dout.release();
    m->dZ3.release();
    m->dpool.release();
    m->parts.release();
    (void)cudaGetLastError();
    delete m;
}

size_t vbh_ws_num_params(const vbh_ws *m) { return m ? m->np : 0; }

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
    int rc = pack(m);
    if (rc) return rc;
    WS_CK(cudaStreamSynchronize(m->stream));
    m->step = 0;
    return VBH_OK;
}

int vbh_ws_set_norm(vbh_ws *m, const float *mean, const float *std)
{
    if (!m || !mean || !std) return VBH_EINVAL;
    const size_t n = size_t(SMAXW + 1) * P;
    for (size_t i = 0; i < n; ++i)
        if (!(std[i] > 0.0f) || !std::isfinite(mean[i]) || !std::isfinite(std[i])) return VBH_EINVAL;
    m->mean.assign(mean, mean + n);
    m->std.assign(std, std + n);
    return VBH_OK;
}

int vbh_ws_features(vbh_ws *m, const float *r, const float *d, int64_t V, int S, int64_t n, float *x)
{
    if (!m || !r || !d || !x || V < 1 || S < 2 || S > SMAXW || n < 0) return VBH_EINVAL;
    if (n > 0 && n < V && V > (1LL << 36)) return VBH_EINVAL;
    const long long nn = (n > 0 && n < V) ? n : V;
    Guard g(m->device);
    features_f32_kernel<<<grid_for(nn, 256), 256, 0, m->stream>>>(r, d, V, S, nn, x);
    WS_CK(cudaGetLastError());
    WS_CK(cudaStreamSynchronize(m->stream));
    return VBH_OK;
}

int vbh_ws_forward(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V, const int *S,
                   const int64_t *n, float *out)
{
    if (!m || !out) return VBH_EINVAL;
    Guard g(m->device);
    int rc;
    if ((rc = plan_batch(m, B, r, d, V, S, n, false)) || (rc = forward(m, false))) return rc;
    WS_CK(cudaMemcpyAsync(out, m->out.p, sizeof(float) * B * P, cudaMemcpyDeviceToDevice, m->stream));
    return check_err(m);
}

int vbh_ws_loss_grad(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V,
                     const int *S, const int64_t *n, const float *target, const float *weight, double *loss,
                     float *grad)
{
    if (!m || !target || !weight) return VBH_EINVAL;
    Guard g(m->device);
    int rc;
    if ((rc = plan_batch(m, B, r, d, V, S, n, true)) || (rc = backward(m, target, weight, loss))) return rc;
    if (grad) WS_CK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->stream));
    return check_err(m);
}

int vbh_ws_train_step(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V,
                      const int *S, const int64_t *n, const float *target, const float *weight, float lr,
                      double *loss)
{
    if (!m || !target || !weight || !(lr > 0.0f)) return VBH_EINVAL;
    Guard g(m->device);
    int rc;
    if ((rc = plan_batch(m, B, r, d, V, S, n, true)) || (rc = backward(m, target, weight, loss))) return rc;
    m->step += 1;
    const float c1 = float(1.0 - std::pow(0.9, m->step)), c2 = float(1.0 - std::pow(0.999, m->step));
    adam_kernel<<<grid_for((long long)m->np, 256), 256, 0, m->stream>>>(m->np, m->theta, m->grad, m->am, m->av, lr,
                                                                       c1, c2);
    WS_CK(cudaGetLastError());
    if ((rc = pack(m))) return rc;
    return check_err(m);
}

int vbh_ws_predict(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V, const int *S,
                   const vbh_prior *p, vbh_result *init)
{
    if (!m || !init || B < 1) return VBH_EINVAL;
    Guard g(m->device);
    int rc;
    if ((rc = plan_batch(m, B, r, d, V, S, nullptr, false)) || (rc = forward(m, false))) return rc;
    std::vector<float> out(size_t(B) * P);
    WS_CK(cudaMemcpyAsync(out.data(), m->out.p, sizeof(float) * out.size(), cudaMemcpyDeviceToHost, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
    if ((rc = check_err(m))) return rc;
    int first = VBH_OK;
    for (int b = 0; b < B; ++b) {
        const int Sb = S[b], M = Sb - 1;
        vbh_prior pd;
        vbh_prior_default(Sb, &pd);
        const vbh_prior &q = p ? p[b] : pd;
        std::vector<double> t(P);
        for (int i = 0; i < P; ++i) {
            const size_t k = size_t(Sb) * P + i;
            t[i] = double(out[size_t(b) * P + i]) * m->std[k] + m->mean[k];
        }
        vbh_result *o = init + b;
        std::memset(o, 0, sizeof(*o));
        o->S = Sb;
        double sum = 0.0;
        for (int j = 0; j < M; ++j) {
            o->kappa[j] = t[j];
            o->weights[j] = t[j];
            sum += t[j];
        }
        o->weights[M] = 1.0 - sum;
        const double erho = std::exp(t[9]);
        std::vector<double> L(size_t(M) * M, 0.0);
        for (int j = 0; j < M; ++j)
            for (int k = 0; k <= j; ++k) {
                const double v = t[10 + j * (j + 1) / 2 + k];
                L[size_t(j) * M + k] = (k == j) ? std::exp(v) : v;
            }
        const double Vd = double(V[b]);
        o->nu = q.n0 + Vd;
        o->lambda = q.q0 + Vd;
        o->a_rho = q.a0 + 0.5 * Vd;
        o->b_rho = o->a_rho / erho;
        o->rho_mean = erho;
        o->rho_mode = (o->a_rho - 1.0) / o->b_rho;
        bool finite = std::isfinite(erho) && erho > 0.0;
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k) {
                double s = 0.0;
                for (int u = 0; u <= (j < k ? j : k); ++u) s += L[size_t(j) * M + u] * L[size_t(k) * M + u];
                o->W_inv[j * M + k] = o->nu * s;              // W^{-1} = nu Sigma0 (Eq. 28)
                finite = finite && std::isfinite(o->W_inv[j * M + k]);
            }
        for (int j = 0; j < M; ++j) finite = finite && std::isfinite(o->kappa[j]);
        o->status = finite ? VBH_OK : VBH_ENONFINITE;
        if (!finite && first == VBH_OK) first = VBH_ENONFINITE;
    }
    return first;
}

} // extern "C"
