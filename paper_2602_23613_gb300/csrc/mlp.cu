// Learned interpolation weights: features of a coarse edge's local problem, a 3-layer perceptron
// (width 64; FP32, or BF16 storage with FP32 accumulation) with hand-written forward/backward/Adam
// kernels, and the scatter of predicted patch values into P.  The layers are small dense products
// (batch x 194 x 64): plain tiled kernels with FP32 accumulation, deterministic summation order.
#include <cmath>
#include <numeric>
#include <vector>

#include "mlp.cuh"
#include "splitmix.cuh"

namespace amgh {

namespace {

// U(0,1) draw i of the network's stream for a seed
__host__ __device__ inline double draw01(uint64_t seed, uint64_t i) { return splitmix_u01(STREAM_MLP, seed, i); }

__global__ void init_layer_kernel(float* W, int fi, int fo, uint64_t seed, uint64_t off) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)fi * fo) return;
    const double lim = sqrt(6.0 / (fi + fo));
    W[t] = (float)((2.0 * draw01(seed, off + (uint64_t)t) - 1.0) * lim);
}

__device__ __forceinline__ float ldf(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void stf(float* p, int64_t i, float v) { p[i] = v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = __float2bfloat16_rn(in[t]);
}

// C (Mr x N, row-major) = A B (+ bias[col]) (relu), A(i,k) = A[i a_rs + k a_cs], B(k,j) = B[k b_rs + j b_cs];
// operands FP32 or BF16, FP32 accumulation, C stored in its type (BF16: rounded to nearest even)
template <class TA, class TB, class TC, bool RELU>
__global__ void gemm_kernel(int Mr, int N, int K, const TA* __restrict__ A, int64_t a_rs, int64_t a_cs,
                            const TB* __restrict__ B, int64_t b_rs, int64_t b_cs, const float* __restrict__ bias,
                            float* __restrict__ Zout, TC* __restrict__ C) {
    __shared__ float As[16][17];
    __shared__ float Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (row < Mr && ka < K) ? ldf(A, row * a_rs + ka * a_cs) : 0.f;
        Bs[ty][tx] = (kb < K && col < N) ? ldf(B, kb * b_rs + col * b_cs) : 0.f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (row < Mr && col < N) {
        const float z = acc + (bias ? bias[col] : 0.f);
        if (Zout) Zout[(int64_t)row * N + col] = z;
        stf(C, (int64_t)row * N + col, RELU ? fmaxf(z, 0.f) : z);
    }
}

// column sums: one CTA of 256 threads per column, each thread a strided partial sum, then a
// fixed-order tree (deterministic)
// split-K part of C = A B: CTA (x, y, z) forms its 16 x 16 tile over k in [z ks, (z + 1) ks) into
// part[z] (M x N); parts are then summed in z order (deterministic)
template <class TA, class TB>
__global__ void gemm_part_kernel(int Mr, int N, int K, int ks, const TA* __restrict__ A, int64_t a_rs, int64_t a_cs,
                                 const TB* __restrict__ B, int64_t b_rs, int64_t b_cs, float* __restrict__ part) {
    __shared__ float As[16][17];
    __shared__ float Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    const int kb0 = blockIdx.z * ks, kb1 = min(K, kb0 + ks);
    float acc = 0.f;
    for (int k0 = kb0; k0 < kb1; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (row < Mr && ka < kb1) ? ldf(A, row * a_rs + ka * a_cs) : 0.f;
        Bs[ty][tx] = (kb < kb1 && col < N) ? ldf(B, kb * b_rs + col * b_cs) : 0.f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (row < Mr && col < N) part[(int64_t)blockIdx.z * Mr * N + (int64_t)row * N + col] = acc;
}

__global__ void sum_parts_kernel(int nparts, int64_t mn, const float* __restrict__ part, float* __restrict__ C) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mn) return;
    float s = part[t];
    for (int z = 1; z < nparts; ++z) s += part[z * mn + t];
    C[t] = s;
}

__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ D, float* __restrict__ out) {
    __shared__ float red[256];
    const int j = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < rows; r += 256) s += D[(int64_t)r * cols + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

__global__ void relu_back_kernel(int64_t n, const float* __restrict__ Z, float* __restrict__ D) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && !(Z[t] > 0.f)) D[t] = 0.f;
}

// masked squared error over the batch, and dy = 2 (y - t) m / sum(m), in three steps with a
// fixed summation order: per-CTA partial sums (FP64), their sum on one CTA, then dy elementwise
constexpr int LOSS_BLOCKS = 152, LOSS_THREADS = 256;

__global__ void __launch_bounds__(LOSS_THREADS) loss_partial_kernel(int64_t n, const float* __restrict__ Y,
                                                                    const float* __restrict__ T,
                                                                    const float* __restrict__ Mk,
                                                                    double* __restrict__ part) {
    __shared__ double sl[LOSS_THREADS], sm[LOSS_THREADS];
    double l = 0.0, m = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * LOSS_THREADS + threadIdx.x; t < n; t += (int64_t)gridDim.x * LOSS_THREADS) {
        const double e = (double)Y[t] - (double)T[t];
        l += e * e * Mk[t];
        m += Mk[t];
    }
    sl[threadIdx.x] = l;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = LOSS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sl[threadIdx.x] += sl[threadIdx.x + o];
            sm[threadIdx.x] += sm[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sl[0];
        part[2 * blockIdx.x + 1] = sm[0];
    }
}

// out[0] = loss, out[2] = sum of the mask (the normaliser); acc[0] += loss when given
__global__ void __launch_bounds__(LOSS_THREADS) loss_final_kernel(int nparts, const double* __restrict__ part,
                                                                  double* __restrict__ out, double* __restrict__ acc) {
    __shared__ double sl[LOSS_THREADS], sm[LOSS_THREADS];
    double l = 0.0, m = 0.0;
    for (int q = threadIdx.x; q < nparts; q += LOSS_THREADS) {
        l += part[2 * q];
        m += part[2 * q + 1];
    }
    sl[threadIdx.x] = l;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = LOSS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sl[threadIdx.x] += sl[threadIdx.x + o];
            sm[threadIdx.x] += sm[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nrm = sm[0] > 0.0 ? sm[0] : 1.0;
        out[0] = sl[0] / nrm;
        out[2] = nrm;
        if (acc) acc[0] += sl[0] / nrm;   // the epoch's running sum (batches run in stream order)
    }
}

__global__ void loss_grad_kernel(int64_t n, const float* __restrict__ Y, const float* __restrict__ T,
                                 const float* __restrict__ Mk, const double* __restrict__ nrm, float* __restrict__ dY) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dY[t] = (float)(2.0 * ((double)Y[t] - (double)T[t]) * Mk[t] / nrm[0]);
}

__global__ void adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float c1, float c2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float a = 0.9f * m1[t] + 0.1f * gt;
    const float b = 0.999f * m2[t] + 0.001f * gt * gt;
    m1[t] = a;
    m2[t] = b;
    p[t] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
}

__global__ void gather_rows_kernel(int nb, int d, const int32_t* __restrict__ perm, const float* __restrict__ src,
                                   float* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nb * d) return;
    const int r = (int)(t / d), c = (int)(t % d);
    dst[t] = src[(int64_t)perm[r] * d + c];
}

__device__ __forceinline__ int bs_find(const int32_t* a, int lo, int hi, int key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}
__device__ __forceinline__ double a_entry(const int32_t* ptr, const int32_t* idx, const double* val, int r, int c) {
    const int q = bs_find(idx, ptr[r], ptr[r + 1], c);
    return q >= 0 ? val[q] : 0.0;
}
__device__ __forceinline__ float slogf_d(double v) { return (float)copysign(log1p(fabs(v)), v); }

// a warp per coarse edge; lanes over the patch slots
__global__ void features_kernel(const int32_t* __restrict__ Aptr, const int32_t* __restrict__ Aidx,
                                const double* __restrict__ Aval, int c0, int nc, const int32_t* __restrict__ edges4,
                                const int32_t* __restrict__ pptr, const int32_t* __restrict__ pidx,
                                const double* __restrict__ Pval, const int64_t* __restrict__ posP,
                                float* __restrict__ X, float* __restrict__ T, float* __restrict__ Mk) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nc) return;
    const int c = c0 + w;
    const int d1 = edges4[4 * c], s1 = edges4[4 * c + 1], d2 = edges4[4 * c + 2], s2 = edges4[4 * c + 3];
    const int p0 = pptr[c], m = pptr[c + 1] - p0;
    const double a11 = a_entry(Aptr, Aidx, Aval, d1, d1);
    float* xr = X + (int64_t)w * MLP_DIN;
    for (int q = lane; q < MLP_SLOTS; q += 32) {
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, tq = 0.f, mq = 0.f;
        if (q < m) {
            const int g = pidx[p0 + q];
            const double diag = a_entry(Aptr, Aidx, Aval, g, g);
            const double rhs = -(a_entry(Aptr, Aidx, Aval, g, d1) * s1 + a_entry(Aptr, Aidx, Aval, g, d2) * s2);
            double off = 0.0;
            for (int e = Aptr[g]; e < Aptr[g + 1]; ++e) {
                const int h = Aidx[e];
                if (h != g && bs_find(pidx, p0, p0 + m, h) >= 0) off += fabs(Aval[e]);
            }
            f0 = slogf_d(diag / a11);
            f1 = slogf_d(rhs / a11);
            f2 = slogf_d(off / a11);
            mq = 1.f;
            if (Pval) tq = (float)Pval[posP[p0 + q]];
        }
        xr[3 * q] = f0;
        xr[3 * q + 1] = f1;
        xr[3 * q + 2] = f2;
        if (T) T[(int64_t)w * MLP_SLOTS + q] = tq;
        if (Mk) Mk[(int64_t)w * MLP_SLOTS + q] = mq;
    }
    if (lane == 0) {
        xr[3 * MLP_SLOTS] = (float)m / MLP_SLOTS;
        xr[3 * MLP_SLOTS + 1] = slogf_d(a_entry(Aptr, Aidx, Aval, d2, d2) / a11);
    }
}

__global__ void scatter_kernel(int c0, int nc, const int32_t* __restrict__ pptr, const float* __restrict__ Y,
                               const int64_t* __restrict__ posP, const int64_t* __restrict__ posPT,
                               double* __restrict__ Pval, double* __restrict__ PTval) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nc) return;
    const int c = c0 + w;
    const int p0 = pptr[c], m = pptr[c + 1] - p0;
    for (int q = lane; q < m && q < MLP_SLOTS; q += 32) {
        const double v = (double)Y[(int64_t)w * MLP_SLOTS + q];
        Pval[posP[p0 + q]] = v;
        PTval[posPT[p0 + q]] = v;
    }
}

template <bool RELU, class TA, class TB, class TC>
void gemm(int Mr, int N, int K, const TA* A, int64_t a_rs, int64_t a_cs, const TB* B, int64_t b_rs, int64_t b_cs,
          const float* bias, float* Zout, TC* C, cudaStream_t s) {
    dim3 blk(16, 16), grd((N + 15) / 16, (Mr + 15) / 16);
    gemm_kernel<TA, TB, TC, RELU><<<grd, blk, 0, s>>>(Mr, N, K, A, a_rs, a_cs, B, b_rs, b_cs, bias, Zout, C);
    AMGH_LAUNCHED();
}

// a weight gradient C (Mr x N) = A B with the batch as K: split over K in slices of 128 when the
// batch is long enough for the plain tiles to leave most SMs idle
constexpr int KSPLIT_MAX = 8;
template <class TA, class TB>
void gemm_wgrad(MlpNet& net, int Mr, int N, int K, const TA* A, int64_t a_rs, int64_t a_cs, const TB* B,
                int64_t b_rs, int64_t b_cs, float* C, cudaStream_t s) {
    const int nparts = std::min(KSPLIT_MAX, std::max(1, K / 128));
    if (nparts == 1) {
        gemm<false>(Mr, N, K, A, a_rs, a_cs, B, b_rs, b_cs, nullptr, nullptr, C, s);
        return;
    }
    const int ks = ((K + nparts - 1) / nparts + 15) / 16 * 16;
    const int nz = (K + ks - 1) / ks;
    const int64_t mn = (int64_t)Mr * N;
    if ((int64_t)net.kparts.n < nz * mn) net.kparts.alloc((size_t)(nz * mn));
    dim3 blk(16, 16), grd((N + 15) / 16, (Mr + 15) / 16, nz);
    gemm_part_kernel<TA, TB><<<grd, blk, 0, s>>>(Mr, N, K, ks, A, a_rs, a_cs, B, b_rs, b_cs, net.kparts.p);
    sum_parts_kernel<<<(unsigned)((mn + 255) / 256), 256, 0, s>>>(nz, mn, net.kparts.p, C);
    AMGH_LAUNCHED();
}

void to_bf16(const float* in, __nv_bfloat16* out, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, out);
    AMGH_LAUNCHED();
}

// the BF16 copies of the parameters, from the FP32 masters
void refresh_wq(MlpNet& net, cudaStream_t s) {
    if (!net.bf16) return;
    if ((int64_t)net.wq.n < net.count()) net.wq.alloc(net.count());
    to_bf16(net.params.p, net.wq.p, net.count(), s);
}

void ensure_batch(MlpNet& net, int nb) {
    if (nb <= net.batch_cap) return;
    net.batch_cap = nb;
    const size_t w = std::max(net.d_in, std::max(net.width, net.d_out));
    net.bx.alloc((size_t)nb * net.d_in);
    net.bt.alloc((size_t)nb * net.d_out);
    net.bm.alloc((size_t)nb * net.d_out);
    net.z1.alloc((size_t)nb * net.width);
    net.h1.alloc((size_t)nb * net.width);
    net.z2.alloc((size_t)nb * net.width);
    net.h2.alloc((size_t)nb * net.width);
    net.y.alloc((size_t)nb * net.d_out);
    net.dy.alloc((size_t)nb * net.d_out);
    net.dh.alloc((size_t)nb * w);
    net.dz.alloc((size_t)nb * w);
    net.xq.alloc((size_t)nb * net.d_in);
    net.h1q.alloc((size_t)nb * net.width);
    net.h2q.alloc((size_t)nb * net.width);
    net.lossbuf.alloc(3);   // the last batch's loss, the epoch's running sum, the last normaliser
    net.losspart.alloc(2 * LOSS_BLOCKS);
}

}  // namespace

void mlp_init(MlpNet& net, uint64_t seed, cudaStream_t s) {
    net.params.alloc(net.count());
    net.grads.alloc(net.count());
    net.m1.alloc(net.count());
    net.m2.alloc(net.count());
    net.params.zero(s);
    net.m1.zero(s);
    net.m2.zero(s);
    net.adam_t = 0;
    const int fi[3] = {net.d_in, net.width, net.width}, fo[3] = {net.width, net.width, net.d_out};
    const int64_t offs[3] = {net.off_W1(), net.off_W2(), net.off_W3()};
    uint64_t draw = 0;
    for (int l = 0; l < 3; ++l) {
        const int64_t cnt = (int64_t)fi[l] * fo[l];
        init_layer_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(net.params.p + offs[l], fi[l], fo[l], seed, draw);
        AMGH_LAUNCHED();
        draw += (uint64_t)cnt;
    }
}

void mlp_reserve(MlpNet& net, int64_t rows, cudaStream_t s) {
    if (rows <= net.capacity) return;
    int64_t cap = std::max<int64_t>(rows, 2 * net.capacity);
    DevArray<float> X, T, M;
    X.alloc((size_t)cap * net.d_in);
    T.alloc((size_t)cap * net.d_out);
    M.alloc((size_t)cap * net.d_out);
    if (net.nsamples) {
        AMGH_CUDA(cudaMemcpyAsync(X.p, net.X.p, sizeof(float) * net.nsamples * net.d_in, cudaMemcpyDeviceToDevice, s));
        AMGH_CUDA(cudaMemcpyAsync(T.p, net.T.p, sizeof(float) * net.nsamples * net.d_out, cudaMemcpyDeviceToDevice, s));
        AMGH_CUDA(cudaMemcpyAsync(M.p, net.M.p, sizeof(float) * net.nsamples * net.d_out, cudaMemcpyDeviceToDevice, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
    }
    net.X = std::move(X);
    net.T = std::move(T);
    net.M = std::move(M);
    net.capacity = cap;
}

// (BF16: the parameters' copies must be current, see refresh_wq)
static void forward_batch(MlpNet& net, const float* X, int nb, float* Y, cudaStream_t s) {
    const float* P = net.params.p;
    if (net.bf16) {
        const __nv_bfloat16* Q = net.wq.p;
        to_bf16(X, net.xq.p, (int64_t)nb * net.d_in, s);
        gemm<true>(nb, net.width, net.d_in, net.xq.p, net.d_in, 1, Q + net.off_W1(), net.width, 1, P + net.off_b1(),
                   net.z1.p, net.h1q.p, s);
        gemm<true>(nb, net.width, net.width, net.h1q.p, net.width, 1, Q + net.off_W2(), net.width, 1,
                   P + net.off_b2(), net.z2.p, net.h2q.p, s);
        gemm<false>(nb, net.d_out, net.width, net.h2q.p, net.width, 1, Q + net.off_W3(), net.d_out, 1,
                    P + net.off_b3(), nullptr, Y, s);
        return;
    }
    gemm<true>(nb, net.width, net.d_in, X, net.d_in, 1, P + net.off_W1(), net.width, 1, P + net.off_b1(), net.z1.p,
               net.h1.p, s);
    gemm<true>(nb, net.width, net.width, net.h1.p, net.width, 1, P + net.off_W2(), net.width, 1, P + net.off_b2(),
               net.z2.p, net.h2.p, s);
    gemm<false>(nb, net.d_out, net.width, net.h2.p, net.width, 1, P + net.off_W3(), net.d_out, 1, P + net.off_b3(),
                nullptr, Y, s);
}

void mlp_forward(MlpNet& net, const float* X, int64_t n, float* Y, cudaStream_t s) {
    const int chunk = 4096;
    ensure_batch(net, chunk);
    refresh_wq(net, s);
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, n - r0);
        forward_batch(net, X + r0 * net.d_in, nb, Y + r0 * net.d_out, s);
    }
}

double mlp_loss_grad(MlpNet& net, const float* X, const float* T, const float* M, int nb, cudaStream_t s,
                     bool read_loss) {
    ensure_batch(net, nb);
    refresh_wq(net, s);
    forward_batch(net, X, nb, net.y.p, s);
    const int64_t ny = (int64_t)nb * net.d_out;
    loss_partial_kernel<<<LOSS_BLOCKS, LOSS_THREADS, 0, s>>>(ny, net.y.p, T, M, net.losspart.p);
    loss_final_kernel<<<1, LOSS_THREADS, 0, s>>>(LOSS_BLOCKS, net.losspart.p, net.lossbuf.p,
                                                 read_loss ? nullptr : net.lossbuf.p + 1);
    loss_grad_kernel<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(ny, net.y.p, T, M, net.lossbuf.p + 2, net.dy.p);
    AMGH_LAUNCHED();
    float* G = net.grads.p;
    const float* P = net.params.p;
    const int w = net.width;
    if (net.bf16) {
        // the same chain with the operands as the forward pass stored them
        const __nv_bfloat16* Q = net.wq.p;
        gemm_wgrad(net, w, net.d_out, nb, net.h2q.p, 1, w, net.dy.p, net.d_out, 1, G + net.off_W3(), s);
        colsum_kernel<<<net.d_out, 256, 0, s>>>(nb, net.d_out, net.dy.p, G + net.off_b3());
        AMGH_LAUNCHED();
        gemm<false>(nb, w, net.d_out, net.dy.p, net.d_out, 1, Q + net.off_W3(), 1, net.d_out, nullptr, nullptr,
                    net.dh.p, s);
        relu_back_kernel<<<(unsigned)(((int64_t)nb * w + 255) / 256), 256, 0, s>>>((int64_t)nb * w, net.z2.p, net.dh.p);
        AMGH_LAUNCHED();
        gemm_wgrad(net, w, w, nb, net.h1q.p, 1, w, net.dh.p, w, 1, G + net.off_W2(), s);
        colsum_kernel<<<w, 256, 0, s>>>(nb, w, net.dh.p, G + net.off_b2());
        AMGH_LAUNCHED();
        gemm<false>(nb, w, w, net.dh.p, w, 1, Q + net.off_W2(), 1, w, nullptr, nullptr, net.dz.p, s);
        relu_back_kernel<<<(unsigned)(((int64_t)nb * w + 255) / 256), 256, 0, s>>>((int64_t)nb * w, net.z1.p, net.dz.p);
        AMGH_LAUNCHED();
        gemm_wgrad(net, net.d_in, w, nb, net.xq.p, 1, net.d_in, net.dz.p, w, 1, G + net.off_W1(), s);
        colsum_kernel<<<w, 256, 0, s>>>(nb, w, net.dz.p, G + net.off_b1());
        AMGH_LAUNCHED();
        double L = 0.0;
        if (read_loss) {
            AMGH_CUDA(cudaMemcpyAsync(&L, net.lossbuf.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            AMGH_CUDA(cudaStreamSynchronize(s));
        }
        return L;
    }
    // layer 3: dW3 = h2^T dy, db3 = colsum(dy), dh2 = dy W3^T
    gemm_wgrad(net, w, net.d_out, nb, net.h2.p, 1, w, net.dy.p, net.d_out, 1, G + net.off_W3(), s);
    colsum_kernel<<<net.d_out, 256, 0, s>>>(nb, net.d_out, net.dy.p, G + net.off_b3());
    AMGH_LAUNCHED();
    gemm<false>(nb, w, net.d_out, net.dy.p, net.d_out, 1, P + net.off_W3(), 1, net.d_out, nullptr, nullptr, net.dh.p, s);
    relu_back_kernel<<<(unsigned)(((int64_t)nb * w + 255) / 256), 256, 0, s>>>((int64_t)nb * w, net.z2.p, net.dh.p);
    AMGH_LAUNCHED();
    // layer 2: dW2 = h1^T dz2, db2, dh1 = dz2 W2^T
    gemm_wgrad(net, w, w, nb, net.h1.p, 1, w, net.dh.p, w, 1, G + net.off_W2(), s);
    colsum_kernel<<<w, 256, 0, s>>>(nb, w, net.dh.p, G + net.off_b2());
    AMGH_LAUNCHED();
    gemm<false>(nb, w, w, net.dh.p, w, 1, P + net.off_W2(), 1, w, nullptr, nullptr, net.dz.p, s);
    relu_back_kernel<<<(unsigned)(((int64_t)nb * w + 255) / 256), 256, 0, s>>>((int64_t)nb * w, net.z1.p, net.dz.p);
    AMGH_LAUNCHED();
    // layer 1: dW1 = X^T dz1, db1
    gemm_wgrad(net, net.d_in, w, nb, X, 1, net.d_in, net.dz.p, w, 1, G + net.off_W1(), s);
    colsum_kernel<<<w, 256, 0, s>>>(nb, w, net.dz.p, G + net.off_b1());
    AMGH_LAUNCHED();
    double L = 0.0;
    if (read_loss) {
        AMGH_CUDA(cudaMemcpyAsync(&L, net.lossbuf.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        AMGH_CUDA(cudaStreamSynchronize(s));
    }
    return L;
}

void mlp_adam(MlpNet& net, float lr, cudaStream_t s) {
    net.adam_t++;
    const float c1 = 1.f - std::pow(0.9f, (float)net.adam_t), c2 = 1.f - std::pow(0.999f, (float)net.adam_t);
    const int64_t n = net.count();
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, net.params.p, net.grads.p, net.m1.p, net.m2.p, lr, c1, c2);
    AMGH_LAUNCHED();
}

double mlp_epoch(MlpNet& net, int batch, float lr, uint64_t seed, cudaStream_t s) {
    const int64_t N = net.nsamples;
    if (N == 0) return 0.0;
    // Fisher-Yates permutation driven by the network's SplitMix64 stream
    std::vector<int32_t> perm(N);
    std::iota(perm.begin(), perm.end(), 0);
    for (int64_t i = N - 1; i > 0; --i) {
        const int64_t j = (int64_t)(draw01(seed, (uint64_t)(N - 1 - i)) * (double)(i + 1));
        std::swap(perm[i], perm[std::min(j, i)]);
    }
    DevArray<int32_t> dperm;
    dperm.upload(perm, s);
    ensure_batch(net, batch);
    // the batch losses add up on the device; the host reads the sum once, after the epoch
    AMGH_CUDA(cudaMemsetAsync(net.lossbuf.p + 1, 0, sizeof(double), s));
    int nbatches = 0;
    for (int64_t r0 = 0; r0 < N; r0 += batch) {
        const int nb = (int)std::min<int64_t>(batch, N - r0);
        gather_rows_kernel<<<(unsigned)(((int64_t)nb * net.d_in + 255) / 256), 256, 0, s>>>(nb, net.d_in, dperm.p + r0,
                                                                                          net.X.p, net.bx.p);
        gather_rows_kernel<<<(unsigned)(((int64_t)nb * net.d_out + 255) / 256), 256, 0, s>>>(nb, net.d_out, dperm.p + r0,
                                                                                           net.T.p, net.bt.p);
        gather_rows_kernel<<<(unsigned)(((int64_t)nb * net.d_out + 255) / 256), 256, 0, s>>>(nb, net.d_out, dperm.p + r0,
                                                                                           net.M.p, net.bm.p);
        AMGH_LAUNCHED();
        mlp_loss_grad(net, net.bx.p, net.bt.p, net.bm.p, nb, s, false);
        mlp_adam(net, lr, s);
        nbatches++;
    }
    double tot = 0.0;
    AMGH_CUDA(cudaMemcpyAsync(&tot, net.lossbuf.p + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMGH_CUDA(cudaStreamSynchronize(s));
    return tot / nbatches;
}

void launch_mlp_features(const DevCSR& A, int c0, int nc, const int32_t* edges4, const int32_t* patch_ptr,
                         const int32_t* patch_idx, const double* Pval, const int64_t* pos_P, float* X, float* T,
                         float* Mk, cudaStream_t s) {
    if (nc == 0) return;
    features_kernel<<<(unsigned)(((int64_t)nc * 32 + 255) / 256), 256, 0, s>>>(
        A.ptr.p, A.idx.p, A.val.p, c0, nc, edges4, patch_ptr, patch_idx, Pval, pos_P, X, T, Mk);
    AMGH_LAUNCHED();
}

void launch_mlp_scatter(int c0, int nc, const int32_t* patch_ptr, const float* Y, const int64_t* pos_P,
                        const int64_t* pos_PT, double* Pval, double* PTval, cudaStream_t s) {
    if (nc == 0) return;
    scatter_kernel<<<(unsigned)(((int64_t)nc * 32 + 255) / 256), 256, 0, s>>>(c0, nc, patch_ptr, Y, pos_P, pos_PT, Pval,
                                                                            PTval);
    AMGH_LAUNCHED();
}

}  // namespace amgh
