// Learned skip proposal: per-vertex features, a 8 -> 32 -> 1 perceptron with
// float16 inputs and weights and float32 accumulation on the ALUs (no tensor
// cores: 288 multiply-adds per vertex are far from a dense contraction), its
// gradient of the mean binary cross-entropy, an Adam step, and the skip
// masks (learned and the "no neighbour moved" rule).  The paper has no
// learned component; this predicts which vertices will not move in the coming
// sweep so that the sweep can skip them.
#include <cuda_fp16.h>

#include "cd_internal.cuh"

namespace cdk {

// Features (float16, 8 per vertex):
//   0 log2(1 + deg) / 16      1 moved in the previous sweep
//   2 min(sweeps since last move, 8) / 8
//   3 log2(1 + |community|) / 24       4 sqrt(Sigma_d / 2m)
//   5 K_i / Sigma_d                     6 K_{i->C_i} / K_i at the vertex's last
//   decision (0 before it)              7 1
__device__ __forceinline__ uint4 vertex_features(int64_t i, const int64_t* __restrict__ off,
                                                 const uint64_t* __restrict__ K, const uint32_t* __restrict__ labels,
                                                 const uint64_t* __restrict__ Sigma, const uint32_t* __restrict__ size,
                                                 unsigned long long two_m, const uint8_t* __restrict__ moved_last,
                                                 const uint8_t* __restrict__ since_move,
                                                 const float* __restrict__ attach, bool attach_raw) {
    const uint32_t d = labels[i];
    const float deg = (float)(off[i + 1] - off[i]);
    const float sd = (float)Sigma[d];
    float f[8];
    f[0] = log2f(1.0f + deg) / 16.0f;
    f[1] = moved_last ? (float)moved_last[i] : 0.0f;
    f[2] = since_move ? fminf((float)since_move[i], 8.0f) / 8.0f : 0.0f;
    f[3] = log2f(1.0f + (float)size[d]) / 24.0f;
    f[4] = two_m ? sqrtf(sd / (float)two_m) : 0.0f;
    f[5] = sd > 0.0f ? (float)K[i] / sd : 0.0f;
    // attach: the ratio, or (attach_raw) K_{i->C_i} as the sweep kernels store it
    const float ki = (float)K[i];
    f[6] = !attach ? 0.0f : !attach_raw ? attach[i] : (K[i] ? attach[i] / ki : 0.0f);
    f[7] = 1.0f;
    uint4 raw;
    __half2* h = reinterpret_cast<__half2*>(&raw);
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = __floats2half2_rn(f[2 * q], f[2 * q + 1]);
    return raw;
}

__global__ void k_features(const int64_t* __restrict__ off, const uint64_t* __restrict__ K,
                           const uint32_t* __restrict__ labels, const uint64_t* __restrict__ Sigma,
                           const uint32_t* __restrict__ size, unsigned long long two_m,
                           const uint8_t* __restrict__ moved_last, const uint8_t* __restrict__ since_move,
                           const float* __restrict__ attach, bool attach_raw, int64_t n,
                           __half* __restrict__ x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    *reinterpret_cast<uint4*>(x + i * 8) =
        vertex_features(i, off, K, labels, Sigma, size, two_m, moved_last, since_move, attach, attach_raw);
}

__device__ __forceinline__ float mlp_logit_raw(const uint4 raw, const float* W1, const float* b1, const float* w2,
                                               float b2, float* h_out) {
    const __half2* hx = reinterpret_cast<const __half2*>(&raw);
    float x[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 v = __half22float2(hx[q]);
        x[2 * q] = v.x;
        x[2 * q + 1] = v.y;
    }
    float z = b2;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
        float a = b1[j];
#pragma unroll
        for (int q = 0; q < 8; ++q) a = fmaf(W1[j * 8 + q], x[q], a);
        a = fmaxf(a, 0.0f);
        if (h_out) h_out[j] = a;
        z = fmaf(w2[j], a, z);
    }
    return z;
}

__device__ __forceinline__ float mlp_logit(const __half* __restrict__ xrow, const float* W1, const float* b1,
                                           const float* w2, float b2, float* h_out) {
    return mlp_logit_raw(*reinterpret_cast<const uint4*>(xrow), W1, b1, w2, b2, h_out);
}

// Parameters (float32 master, device): W1 [0, 256), b1 [256, 288), w2 [288, 320),
// b2 [320].  The multiply weights W1 and w2 are rounded to float16 as they are
// staged in shared memory; biases and accumulation stay float32.
constexpr int kGradLen = 32 * 8 + 32 + 32 + 1;

__device__ __forceinline__ void load_weights(const float* __restrict__ param, float* W1, float* b1, float* w2,
                                             float* b2) {
    for (int t = threadIdx.x; t < 32 * 8; t += blockDim.x) W1[t] = __half2float(__float2half_rn(param[t]));
    for (int t = threadIdx.x; t < 32; t += blockDim.x) {
        b1[t] = param[256 + t];
        w2[t] = __half2float(__float2half_rn(param[288 + t]));
    }
    if (threadIdx.x == 0) *b2 = param[320];
    __syncthreads();
}

// p[i] = sigmoid(z_i); if thr_active, active[i] = (p[i] >= thr) (the skip mask).
__global__ void k_mlp_forward(const __half* __restrict__ x, int64_t n, const float* __restrict__ param,
                              float* __restrict__ p, uint8_t* __restrict__ active, float thr) {
    __shared__ float W1[256], b1[32], w2[32], b2;
    load_weights(param, W1, b1, w2, &b2);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float z = mlp_logit(x + i * 8, W1, b1, w2, b2, nullptr);
    const float pi = 1.0f / (1.0f + expf(-z));
    if (p) p[i] = pi;
    if (active) active[i] = pi >= thr ? 1 : 0;
}

// The driver's skip proposal in one pass: the features of k_features and the
// forward pass of k_mlp_forward on them (same float16 rounding and float32
// arithmetic, so the same mask), without the feature rows in memory.
__global__ void k_propose(const int64_t* __restrict__ off, const uint64_t* __restrict__ K,
                          const uint32_t* __restrict__ labels, const uint64_t* __restrict__ Sigma,
                          const uint32_t* __restrict__ size, unsigned long long two_m,
                          const uint8_t* __restrict__ moved_last, const uint8_t* __restrict__ since_move,
                          const float* __restrict__ attach, int64_t n, const float* __restrict__ param, float thr,
                          uint8_t* __restrict__ active) {
    __shared__ float W1[256], b1[32], w2[32], b2;
    load_weights(param, W1, b1, w2, &b2);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 raw = vertex_features(i, off, K, labels, Sigma, size, two_m, moved_last, since_move, attach, true);
    const float z = mlp_logit_raw(raw, W1, b1, w2, b2, nullptr);
    const float pi = 1.0f / (1.0f + expf(-z));
    active[i] = pi >= thr ? 1 : 0;
}

// Per-block partial gradients of sum_i BCE(p_i, y_i) (321 floats per block,
// parameter order), in a fixed order: the block's 256 samples store their
// hidden activations and dz = p - y in shared memory, then each parameter's
// sum over the samples is taken by one thread in sample order.

__global__ void __launch_bounds__(256) k_mlp_grad(const __half* __restrict__ x, const uint8_t* __restrict__ y,
                                                  int64_t n, const float* __restrict__ param,
                                                  float* __restrict__ partial, float* __restrict__ loss_partial) {
    __shared__ float W1[256], b1[32], w2[32], b2;
    __shared__ float hs[256][33];
    __shared__ float xs[256][8];
    __shared__ float dzs[256];
    __shared__ float lsum[256];
    load_weights(param, W1, b1, w2, &b2);
    const int t = threadIdx.x;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + t;
    float l = 0.0f, dz = 0.0f;
    float h[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) h[j] = 0.0f;
    float xv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < n) {
        const float z = mlp_logit(x + i * 8, W1, b1, w2, b2, h);
        const float yi = (float)y[i];
        const float pi = 1.0f / (1.0f + expf(-z));
        l = fmaxf(z, 0.0f) - z * yi + log1pf(expf(-fabsf(z)));
        dz = pi - yi;
        const uint4 raw = *reinterpret_cast<const uint4*>(x + i * 8);
        const __half2* hx = reinterpret_cast<const __half2*>(&raw);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 v = __half22float2(hx[q]);
            xv[2 * q] = v.x;
            xv[2 * q + 1] = v.y;
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) hs[t][j] = h[j];
#pragma unroll
    for (int q = 0; q < 8; ++q) xs[t][q] = xv[q];
    dzs[t] = dz;
    lsum[t] = l;
    __syncthreads();
    for (int pidx = t; pidx < kGradLen; pidx += blockDim.x) {
        float acc = 0.0f;
        if (pidx < 256) {
            const int j = pidx / 8, q = pidx % 8;
            for (int s2 = 0; s2 < 256; ++s2)
                if (hs[s2][j] > 0.0f) acc = fmaf(dzs[s2] * w2[j], xs[s2][q], acc);
        } else if (pidx < 288) {
            const int j = pidx - 256;
            for (int s2 = 0; s2 < 256; ++s2)
                if (hs[s2][j] > 0.0f) acc += dzs[s2] * w2[j];
        } else if (pidx < 320) {
            const int j = pidx - 288;
            for (int s2 = 0; s2 < 256; ++s2) acc = fmaf(dzs[s2], hs[s2][j], acc);
        } else {
            for (int s2 = 0; s2 < 256; ++s2) acc += dzs[s2];
        }
        partial[(int64_t)blockIdx.x * kGradLen + pidx] = acc;
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o >= 1; o >>= 1) {
        if (t < o) lsum[t] += lsum[t + o];
        __syncthreads();
    }
    if (t == 0) loss_partial[blockIdx.x] = lsum[0];
}

// Sums the block partials and divides by n: block p takes parameter p (the
// last block the loss); thread t adds the partials of blocks t, t + 256, ...
// in that order, then the 256 sums are added by a fixed tree.  The order of
// every addition is fixed, so the result is the same on every run.
__global__ void __launch_bounds__(256) k_mlp_grad_sum(const float* __restrict__ partial,
                                                      const float* __restrict__ loss_partial, int64_t nblocks,
                                                      int64_t n, float* __restrict__ grad, float* __restrict__ loss) {
    __shared__ double sh[256];
    const int p = blockIdx.x;  // 0 .. kGradLen (kGradLen = the loss)
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t b = t; b < nblocks; b += 256) s += p < kGradLen ? partial[b * kGradLen + p] : loss_partial[b];
    sh[t] = s;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    if (t == 0) {
        if (p < kGradLen) grad[p] = (float)(sh[0] / (double)n);
        else *loss = (float)(sh[0] / (double)n);
    }
}

// Adam step on the float32 master parameters (param layout as the gradient).
__global__ void k_adam(float* __restrict__ param, const float* __restrict__ grad, float* __restrict__ m1,
                       float* __restrict__ m2, int step, float lr) {
    const int t = threadIdx.x;
    if (t >= kGradLen) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gr = grad[t];
    m1[t] = b1 * m1[t] + (1.0f - b1) * gr;
    m2[t] = b2 * m2[t] + (1.0f - b2) * gr * gr;
    const float mh = m1[t] / (1.0f - powf(b1, (float)step));
    const float vh = m2[t] / (1.0f - powf(b2, (float)step));
    param[t] -= lr * mh / (sqrtf(vh) + eps);
}

// moved_last[i] = labels changed; since_move updated (saturating at 255).
__global__ void k_move_state(const uint32_t* __restrict__ before, const uint32_t* __restrict__ after, int64_t n,
                             uint8_t* __restrict__ moved_last, uint8_t* __restrict__ since_move) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool mv = before[i] != after[i];
    moved_last[i] = mv ? 1 : 0;
    const uint8_t s = since_move[i];
    since_move[i] = mv ? 0 : (s < 255 ? s + 1 : 255);
}

// "No neighbour moved" rule: active[j] = 1 for every mover and every
// neighbour of a mover (scatter from the mover list of the last sweep).
__global__ void k_mark_neighbours(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                                  const uint32_t* __restrict__ movers, const Globals* __restrict__ glob,
                                  uint8_t* __restrict__ active) {
    const unsigned long long cnt = glob->moved;
    for (unsigned long long t = blockIdx.x; t < cnt; t += gridDim.x) {
        const uint32_t i = movers[t];
        if (threadIdx.x == 0) active[i] = 1;
        for (int64_t e = off[i] + threadIdx.x; e < off[i + 1]; e += blockDim.x) active[cols[e]] = 1;
    }
}

// ---- launchers ---------------------------------------------------------------------------

cudaError_t launch_features(const int64_t* off, const uint64_t* K, const uint32_t* labels, const uint64_t* Sigma,
                            const uint32_t* size, unsigned long long two_m, const uint8_t* moved_last,
                            const uint8_t* since_move, const float* attach, bool attach_raw, int64_t n, void* x,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_features<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(off, K, labels, Sigma, size, two_m, moved_last,
                                                           since_move, attach, attach_raw, n,
                                                           static_cast<__half*>(x));
    return cudaGetLastError();
}

cudaError_t launch_propose(const int64_t* off, const uint64_t* K, const uint32_t* labels, const uint64_t* Sigma,
                           const uint32_t* size, unsigned long long two_m, const uint8_t* moved_last,
                           const uint8_t* since_move, const float* attach, int64_t n, const float* param, float thr,
                           uint8_t* active, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_propose<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(off, K, labels, Sigma, size, two_m, moved_last, since_move,
                                                          attach, n, param, thr, active);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* x, int64_t n, const float* param, float* p, uint8_t* active, float thr,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_mlp_forward<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(static_cast<const __half*>(x), n, param, p, active,
                                                              thr);
    return cudaGetLastError();
}

int64_t mlp_grad_blocks(int64_t n) { return (n + 255) / 256; }
int mlp_param_count() { return kGradLen; }

// partial: mlp_grad_blocks(n) * 321 floats, loss_partial: mlp_grad_blocks(n).
cudaError_t launch_mlp_grad(const void* x, const uint8_t* y, int64_t n, const float* param, float* partial,
                            float* loss_partial, float* grad, float* loss, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t nb = mlp_grad_blocks(n);
    note_launch();
    k_mlp_grad<<<(unsigned)nb, 256, 0, s>>>(static_cast<const __half*>(x), y, n, param, partial, loss_partial);
    note_launch();
    k_mlp_grad_sum<<<kGradLen + 1, 256, 0, s>>>(partial, loss_partial, nb, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* param, const float* grad, float* m1, float* m2, int step, float lr, cudaStream_t s) {
    note_launch();
    k_adam<<<1, 352, 0, s>>>(param, grad, m1, m2, step, lr);
    return cudaGetLastError();
}

cudaError_t launch_move_state(const uint32_t* before, const uint32_t* after, int64_t n, uint8_t* moved_last,
                              uint8_t* since_move, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_move_state<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(before, after, n, moved_last, since_move);
    return cudaGetLastError();
}

cudaError_t launch_mark_neighbours(const int64_t* off, const int32_t* cols, const uint32_t* movers,
                                   const Globals* glob, uint8_t* active, cudaStream_t s) {
    note_launch();
    k_mark_neighbours<<<152 * 16, 128, 0, s>>>(off, cols, movers, glob, active);
    return cudaGetLastError();
}

// Trace sampling: flags[i] = 1 for the vertices with edges picked by the hash
// of (i, sweep) at rate thr32 / 2^32; the samples are then written in vertex
// order at the exclusive prefix sum of the flags (deterministic order).
__global__ void k_trace_flags(const int64_t* __restrict__ off, int64_t n, int sweep, uint32_t thr32,
                              uint32_t* __restrict__ flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t h = (uint32_t)i ^ ((uint32_t)sweep * 0x9E3779B9u);
    h ^= h >> 16; h *= 0x7feb352dU; h ^= h >> 15; h *= 0x846ca68bU; h ^= h >> 16;
    flags[i] = (off[i + 1] > off[i] && h < thr32) ? 1u : 0u;
}

__global__ void k_trace_write(const __half* __restrict__ x, const uint8_t* __restrict__ moved_last,
                              const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos, int64_t n,
                              int64_t base, __half* __restrict__ xo, uint8_t* __restrict__ yo, int64_t cap) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    const int64_t slot = base + pos[i];
    if (slot >= cap) return;
    *reinterpret_cast<uint4*>(xo + slot * 8) = *reinterpret_cast<const uint4*>(x + i * 8);
    yo[slot] = moved_last[i];
}

cudaError_t launch_trace_flags(const int64_t* off, int64_t n, int sweep, uint32_t thr32, uint32_t* flags,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_trace_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(off, n, sweep, thr32, flags);
    return cudaGetLastError();
}

cudaError_t launch_trace_write(const void* x, const uint8_t* moved_last, const uint32_t* flags, const uint32_t* pos,
                               int64_t n, int64_t base, void* xo, uint8_t* yo, int64_t cap, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    k_trace_write<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(static_cast<const __half*>(x), moved_last, flags, pos,
                                                              n, base, static_cast<__half*>(xo), yo, cap);
    return cudaGetLastError();
}

}  // namespace cdk
