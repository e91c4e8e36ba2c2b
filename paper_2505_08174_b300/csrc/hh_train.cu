// hh_train.cu -- training the pair MLP on the GPU (Section 2.3, Eq. 5).
//
// Samples are two-particle configurations: separation r_s (particle 1 minus
// particle 2), unit force e_s on particle 2, teacher velocity U_s of particle
// 1 (given, or the closed-form RPY velocity K_RPY(r_s) e_s when no teacher
// array is passed -- the stand-in for the paper's Stokesian-dynamics data).
// The surrogate velocity is K(r_s) e_s with K = S(MLP(f)) / |r| (Eq. 4).
//   L = (1/B) sum_s |U_s - K(r_s) e_s|^2 / |U_s|^2                 (Eq. 5)
//
// k_train_sample: one thread per sample -- forward pass (activations kept in
//   registers), loss term, reverse pass to the pre-activation cotangents of
//   every layer; writes the layer inputs H_l and cotangents G_l per sample.
// k_train_wgrad:  one thread per parameter -- dW_l[o][i] = sum_s G_l[s][o]
//   H_l[s][i], db_l[o] = sum_s G_l[s][o], summed in sample order (the
//   gradient is bit-reproducible).
// k_loss_sum:     ordered reduction of the per-sample loss terms.
// k_adam:         Adam (Kingma & Ba 2015) with bias correction.
#include <algorithm>

#include "hh_internal.h"

namespace {

template <int W>
struct TrainLayout {
    // per-sample record: H0 (4), H1 (W), H2 (W), H3 (W), G1 (W), G2 (W), G3 (W), G4 (6)
    static constexpr int H0 = 0, H1 = 4, H2 = 4 + W, H3 = 4 + 2 * W;
    static constexpr int G1 = 4 + 3 * W, G2 = 4 + 4 * W, G3 = 4 + 5 * W, G4 = 4 + 6 * W;
    static constexpr int REC = 4 + 6 * W + 6;
};

__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + __expf(-x)); }

template <int W>
__global__ void __launch_bounds__(128) k_train_sample(const float* __restrict__ th, const double* __restrict__ r,
                                                      const double* __restrict__ e, const double* __restrict__ U,
                                                      int64_t B, float a, float* __restrict__ rec,
                                                      float* __restrict__ loss)
{
    using L = TrainLayout<W>;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float* W1 = th;
    const float* b1 = W1 + 4 * W;
    const float* W2 = b1 + W;
    const float* b2 = W2 + W * W;
    const float* W3 = b2 + W;
    const float* b3 = W3 + W * W;
    const float* W4 = b3 + W;
    const float* b4 = W4 + 6 * W;
    float* R = rec + s * L::REC;

    const float rx = (float)r[3 * s], ry = (float)r[3 * s + 1], rz = (float)r[3 * s + 2];
    const float ex = (float)e[3 * s], ey = (float)e[3 * s + 1], ez = (float)e[3 * s + 2];
    const float id = rsqrtf(rx * rx + ry * ry + rz * rz);
    float f[4] = {rx * id, ry * id, rz * id, a * id};
    float u[3];
    if (U) {
        u[0] = (float)U[3 * s]; u[1] = (float)U[3 * s + 1]; u[2] = (float)U[3 * s + 2];
    } else {  // RPY teacher, mu = 1
        const float d = 1.0f / id;
        float A, Bc;
        if (d >= 2.f * a) {
            const float c = (float)(1.0 / (8.0 * HH_PI)) * id;
            A = c * (1.f + (2.f / 3.f) * a * a * id * id);
            Bc = c * (1.f - 2.f * a * a * id * id);
        } else {
            const float c = (float)(1.0 / (6.0 * HH_PI)) / a;
            A = c * (1.f - (9.f / 32.f) * d / a);
            Bc = c * ((3.f / 32.f) * d / a);
        }
        const float fe = f[0] * ex + f[1] * ey + f[2] * ez;
        u[0] = A * ex + Bc * f[0] * fe;
        u[1] = A * ey + Bc * f[1] * fe;
        u[2] = A * ez + Bc * f[2] * fe;
    }
    // forward (pre-activations z, activations a)
    float z1[W], z2[W], z3[W], a1[W], a2[W], h[W];
    for (int j = 0; j < W; ++j) {
        float t = b1[j];
        for (int i = 0; i < 4; ++i) t += W1[4 * j + i] * f[i];
        z1[j] = t;
        a1[j] = silu_f(t);
    }
    for (int j = 0; j < W; ++j) {
        float t = b2[j];
        for (int i = 0; i < W; ++i) t += W2[W * j + i] * a1[i];
        z2[j] = t;
        a2[j] = silu_f(t);
    }
    for (int j = 0; j < W; ++j) {
        float t = b3[j];
        for (int i = 0; i < W; ++i) t += W3[W * j + i] * a2[i];
        z3[j] = t;
        h[j] = silu_f(t);
    }
    float o[6];
    for (int j = 0; j < 6; ++j) {
        float t = b4[j];
        for (int i = 0; i < W; ++i) t += W4[W * j + i] * h[i];
        o[j] = t;
    }
    // K e = S(o) e / d;  residual, loss term
    const float ke0 = (o[0] * ex + o[3] * ey + o[4] * ez) * id;
    const float ke1 = (o[3] * ex + o[1] * ey + o[5] * ez) * id;
    const float ke2 = (o[4] * ex + o[5] * ey + o[2] * ez) * id;
    const float res[3] = {ke0 - u[0], ke1 - u[1], ke2 - u[2]};
    const float nu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    loss[s] = (res[0] * res[0] + res[1] * res[1] + res[2] * res[2]) / nu;
    // reverse: dL/d(Ke) = 2 res / (B |U|^2); dL/dS_ab = g_a e_b / d; o -> S pattern
    const float sc = 2.0f / ((float)B * nu);
    const float g[3] = {sc * res[0], sc * res[1], sc * res[2]};
    const float e3[3] = {ex, ey, ez};
    float G[9];
    for (int aa = 0; aa < 3; ++aa)
        for (int bb = 0; bb < 3; ++bb) G[3 * aa + bb] = g[aa] * e3[bb] * id;
    float go[6] = {G[0], G[4], G[8], G[1] + G[3], G[2] + G[6], G[5] + G[7]};
    // record layer inputs and the output cotangent
    for (int i = 0; i < 4; ++i) R[L::H0 + i] = f[i];
    for (int i = 0; i < W; ++i) {
        R[L::H1 + i] = a1[i];
        R[L::H2 + i] = a2[i];
        R[L::H3 + i] = h[i];
    }
    for (int j = 0; j < 6; ++j) R[L::G4 + j] = go[j];
    // dL/dz3 = (W4^T go) * silu'(z3)
    float gz[W];
    for (int i = 0; i < W; ++i) {
        float t = 0.f;
        for (int j = 0; j < 6; ++j) t += W4[W * j + i] * go[j];
        const float sg = sigmoid_f(z3[i]);
        gz[i] = t * sg * (1.f + z3[i] * (1.f - sg));
        R[L::G3 + i] = gz[i];
    }
    float gy[W];
#pragma unroll 4
    for (int i = 0; i < W; ++i) {
        float t = 0.f;
        for (int j = 0; j < W; ++j) t += W3[W * j + i] * gz[j];
        const float sg = sigmoid_f(z2[i]);
        gy[i] = t * sg * (1.f + z2[i] * (1.f - sg));
        R[L::G2 + i] = gy[i];
    }
#pragma unroll 4
    for (int i = 0; i < W; ++i) {
        float t = 0.f;
        for (int j = 0; j < W; ++j) t += W2[W * j + i] * gy[j];
        const float sg = sigmoid_f(z1[i]);
        R[L::G1 + i] = t * sg * (1.f + z1[i] * (1.f - sg));
    }
}

// One thread per parameter.  Layer l: inputs H_l (ni) and cotangents G_l (no).
template <int W>
__global__ void k_train_wgrad(const float* __restrict__ rec, int64_t B, float* __restrict__ grad)
{
    using L = TrainLayout<W>;
    const int dims[5] = {4, W, W, W, 6};
    const int hoff[4] = {L::H0, L::H1, L::H2, L::H3};
    const int goff[4] = {L::G1, L::G2, L::G3, L::G4};
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int base = 0;
    for (int l = 0; l < 4; ++l) {
        const int ni = dims[l], no = dims[l + 1], nl = ni * no + no;
        if (x < nl) {
            const int o = x < ni * no ? x / ni : x - ni * no;
            const int i = x < ni * no ? x % ni : -1;
            float acc = 0.f;
            for (int64_t s = 0; s < B; ++s) {
                const float* R = rec + s * L::REC;
                acc += R[goff[l] + o] * (i >= 0 ? R[hoff[l] + i] : 1.0f);
            }
            grad[base + x] = acc;
            return;
        }
        x -= nl;
        base += nl;
    }
}

__global__ void k_loss_sum(const float* __restrict__ loss, int64_t B, double* __restrict__ out)
{
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) acc += (double)loss[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / (double)B;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// Loss (host, FP64) and gradient (grad_dev, float32, may be NULL) of Eq. 5.
double train_loss_grad(hh_ctx* ctx, const float* theta, int width, const double* r, const double* e, const double* U,
                       int64_t B, double a, float* grad_dev, cudaStream_t s)
{
    (void)ctx;
    HH_REQUIRE(width == 32 || width == 64, HH_ERR_ARG, "width must be 32 or 64");
    HH_REQUIRE(B >= 1, HH_ERR_ARG, "batch must be >= 1");
    const int rec_n = width == 32 ? TrainLayout<32>::REC : TrainLayout<64>::REC;
    float* rec = dev_alloc_t<float>(B * rec_n, s);
    float* loss = dev_alloc_t<float>(B, s);
    double* dl = dev_alloc_t<double>(1, s);
    const unsigned g1 = (unsigned)ceil_div(B, 128);
    if (width == 32) k_train_sample<32><<<g1, 128, 0, s>>>(theta, r, e, U, B, (float)a, rec, loss);
    else k_train_sample<64><<<g1, 128, 0, s>>>(theta, r, e, U, B, (float)a, rec, loss);
    HH_CHECK_LAUNCH();
    if (grad_dev) {
        const int P = 4 * width + width + 2 * (width * width + width) + 6 * width + 6;
        if (width == 32) k_train_wgrad<32><<<(unsigned)ceil_div(P, 128), 128, 0, s>>>(rec, B, grad_dev);
        else k_train_wgrad<64><<<(unsigned)ceil_div(P, 128), 128, 0, s>>>(rec, B, grad_dev);
        HH_CHECK_LAUNCH();
    }
    k_loss_sum<<<1, 256, 0, s>>>(loss, B, dl);
    HH_CHECK_LAUNCH();
    double h = 0.0;
    HH_CUDA(cudaMemcpyAsync(&h, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
    HH_CUDA(cudaStreamSynchronize(s));
    dev_free(rec, s);
    dev_free(loss, s);
    dev_free(dl, s);
    return h;
}

void adam_step(float* theta, const float* g, float* m, float* v, int n, int64_t t, double lr, double b1, double b2,
               double eps, cudaStream_t s)
{
    HH_REQUIRE(t >= 1, HH_ERR_ARG, "Adam step count starts at 1");
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    k_adam<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(theta, g, m, v, n, (float)lr, (float)b1, (float)b2, (float)eps,
                                                       (float)c1, (float)c2);
    HH_CHECK_LAUNCH();
}
