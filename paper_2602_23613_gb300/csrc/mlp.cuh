// Learned interpolation weights: a 3-layer perceptron (width 64, FP32, or BF16 storage of inputs,
// weights and hidden activations with FP32 accumulation) that maps a finest-level coarse edge's
// local problem to the values of its column of P on the patch (the interior part of Eq. sparseP),
// with our own forward, backward and Adam kernels.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace amgh {

constexpr int MLP_SLOTS = 64;                     // patch slots (larger patches fall back to solves)
constexpr int MLP_DIN = 3 * MLP_SLOTS + 2;        // features per coarse edge
constexpr int MLP_WIDTH = 64;

struct MlpNet {
    int d_in = MLP_DIN, width = MLP_WIDTH, d_out = MLP_SLOTS;
    DevArray<float> params, grads, m1, m2;        // W1, b1, W2, b2, W3, b3 (row-major W: in x out)
    int64_t adam_t = 0;
    DevArray<float> X, T, M;                      // training samples (capacity rows)
    int64_t nsamples = 0, capacity = 0;
    DevArray<float> bx, bt, bm, z1, h1, z2, h2, y, dy, dh, dz;   // batch buffers
    int batch_cap = 0;
    // BF16 storage: the products read bfloat16 copies of the inputs (xq), of the parameters (wq,
    // refreshed from the FP32 masters before every pass) and of the hidden activations (h1q,
    // h2q); accumulation, biases, outputs, gradients and Adam stay FP32
    bool bf16 = false;
    DevArray<__nv_bfloat16> wq, xq, h1q, h2q;
    DevArray<double> lossbuf, losspart;
    DevArray<float> kparts;                       // split-K parts of the weight gradients
    int64_t off_W1() const { return 0; }
    int64_t off_b1() const { return (int64_t)d_in * width; }
    int64_t off_W2() const { return off_b1() + width; }
    int64_t off_b2() const { return off_W2() + (int64_t)width * width; }
    int64_t off_W3() const { return off_b2() + width; }
    int64_t off_b3() const { return off_W3() + (int64_t)width * d_out; }
    int64_t count() const { return off_b3() + d_out; }
};

// Glorot-uniform initial weights from the SplitMix64 stream (stream 7, seed), zero biases
void mlp_init(MlpNet& net, uint64_t seed, cudaStream_t s);
// forward pass for n rows of X (n x d_in) into Y (n x d_out); uses the batch buffers in chunks
void mlp_forward(MlpNet& net, const float* X, int64_t n, float* Y, cudaStream_t s);
// loss and gradients of a batch (X, T, M device arrays of nb rows) into net.grads; returns the loss
// (read_loss = false: returns 0 without waiting and adds the loss to the epoch sum, lossbuf[1])
double mlp_loss_grad(MlpNet& net, const float* X, const float* T, const float* M, int nb, cudaStream_t s,
                     bool read_loss = true);
void mlp_adam(MlpNet& net, float lr, cudaStream_t s);
// one pass over the sample set in shuffled batches (permutation from stream 7 with the epoch seed)
double mlp_epoch(MlpNet& net, int batch, float lr, uint64_t seed, cudaStream_t s);
void mlp_reserve(MlpNet& net, int64_t rows, cudaStream_t s);

// features (nc x MLP_DIN), targets and masks of coarse edges [c0, c0 + nc) from A (FP64 CSR), the
// edges (4 ints each), the sorted patches and, when Pval/pos are given, the exact P values
void launch_mlp_features(const DevCSR& A, int c0, int nc, const int32_t* edges4, const int32_t* patch_ptr,
                         const int32_t* patch_idx, const double* Pval, const int64_t* pos_P, float* X, float* T,
                         float* Mk, cudaStream_t s);
// scatter predicted patch values (nc x MLP_SLOTS) into P and P^T
void launch_mlp_scatter(int c0, int nc, const int32_t* patch_ptr, const float* Y, const int64_t* pos_P,
                        const int64_t* pos_PT, double* Pval, double* PTval, cudaStream_t s);

}  // namespace amgh
