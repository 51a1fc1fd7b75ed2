// Learned surrogate: a 3D spectral neural operator (forward, backward, Adam) and the
// surrogate-first photoionization solve with the FMM as judge and fallback.
//
// Network on an n^3 grid, width C, m modes per axis, L layers, projection width P:
//   v_0 = Wl u + bl;  z_l = SpecConv_l(v_l) + W_l v_l + b_l;  v_{l+1} = GELU(z_l) (l < L-1),
//   v_L = z_{L-1};  y = Q2 . GELU(Q1 v_L + q1) + q2,
//   SpecConv(v)(o, x) = (1/n^3) sum_{k in K} w_kz Re[ (R(k) V(k))_o e^{+2 pi i k.x/n} ],
//   V(c, k) = sum_x v(c, x) e^{-2 pi i k.x/n},  K = Kx x Ky x Kz,
//   Kx = Ky = {0..m-1} U {n-m..n-1}, Kz = {0..m-1}, w_0 = 1, w_{kz>=1} = 2.
// The truncated transforms are done axis by axis as small dense DFTs against twiddle
// tables (a partial DFT keeps 2m of n frequencies, so a full FFT would be wasted work).
// Spectral weights R are held in FP32 (master) and used rounded to BF16 (FP32
// accumulation) unless the model is switched to FP32 weights.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "kernel.cuh"

namespace kifmm {

struct SnoModel {
    int n = 64, C = 32, m = 12, L = 4, P = 64, maxB = 32;
    int bf16 = 1;
    cudaStream_t st = nullptr;
    int64_t K = 0, np3 = 0;          // modes, grid points
    int64_t nparam = 0;
    std::vector<int64_t> off;        // offsets: Wl, bl, then per layer Rr, Ri, W, b, then Q1, q1, Q2, q2
    DevBuf theta, grad, adam_m, adam_v, rbf;   // rbf: BF16 copies of Rr, Ri per layer
    DevBuf tabs;                     // float2 twiddle tables
    int64_t tzf, tyf, tzb, txi, tzi, tzr;   // table offsets (float2 units)
    // activations (FP32): v[L+1][B][C][np3], z[L][B][C][np3]
    DevBuf v, z, s, cz, cy, cx, g, gx, gy, dv, dz, loss;
    DevBuf ph, pda;                  // projection backward: GELU(a) and dL/da, [B][P][np3]
    DevBuf jt, jref, jorig, jerr;    // photo_solve judge: targets, reference values, caller indices, error
    int64_t steps = 0;
};

// ---- layout ----------------------------------------------------------------------------
static void sno_layout(SnoModel& M) {
    const int64_t C = M.C, K = M.K;
    M.off.clear();
    int64_t o = 0;
    auto add = [&](int64_t k) {
        M.off.push_back(o);
        o += k;
    };
    add(C);
    add(C);
    for (int l = 0; l < M.L; ++l) {
        add(K * C * C);
        add(K * C * C);
        add(C * C);
        add(C);
    }
    add((int64_t)M.P * C);
    add(M.P);
    add(M.P);
    add(1);
    M.nparam = o;
}
enum { O_WL = 0, O_BL = 1 };
static inline int o_rr(int l) { return 2 + 4 * l; }
static inline int o_ri(int l) { return 3 + 4 * l; }
static inline int o_w(int l) { return 4 + 4 * l; }
static inline int o_b(int l) { return 5 + 4 * l; }
static inline int o_q1(const SnoModel& M) { return 2 + 4 * M.L; }

static inline unsigned nbs(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- kernels ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

// Twiddle tables. kind: frequency list for the output (forward) or input (inverse) index.
__global__ void k_tables(int n, int m, float2* t, int64_t tzf, int64_t tyf, int64_t tzb, int64_t txi, int64_t tzi,
                         int64_t tzr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double tw = 6.283185307179586476925286766559 / n;
    const double n3 = (double)n * n * n;
    auto kxy = [&](int k) { return k < m ? k : n - 2 * m + k; };   // index 0..2m-1 -> frequency
    if (i < m * n) {   // tzf[kz][z] = e^{-i kz z}, tzb = (w/n^3) e^{-i kz z}
        int kz = i / n, z = i % n;
        double a = tw * kz * z;
        double w = (kz == 0 ? 1.0 : 2.0) / n3;
        t[tzf + i] = make_float2((float)cos(a), (float)-sin(a));
        t[tzb + i] = make_float2((float)(w * cos(a)), (float)(-w * sin(a)));
    }
    if (i < 2 * m * n) {   // tyf[k][y] = e^{-i ky y}
        int k = i / n, y = i % n;
        double a = tw * kxy(k) * y;
        t[tyf + i] = make_float2((float)cos(a), (float)-sin(a));
    }
    if (i < n * 2 * m) {   // txi[x][k] = e^{+i kx x}
        int x = i / (2 * m), k = i % (2 * m);
        double a = tw * kxy(k) * x;
        t[txi + i] = make_float2((float)cos(a), (float)sin(a));
    }
    if (i < n * m) {   // tzi[z][kz] = (w/n^3) e^{+i kz z}; tzr[z][kz] = e^{+i kz z}
        int z = i / m, kz = i % m;
        double a = tw * kz * z;
        double w = (kz == 0 ? 1.0 : 2.0) / n3;
        t[tzi + i] = make_float2((float)(w * cos(a)), (float)(w * sin(a)));
        t[tzr + i] = make_float2((float)cos(a), (float)sin(a));
    }
}

// out[o][j][i] = sum_q T[j][q] in[o][q][i] along the middle axis (lengths Lin -> Lout),
// in/out real (float) or complex (float2); real output takes the real part.
template <bool CIN, bool COUT>
__global__ void k_dft(const void* __restrict__ in, void* __restrict__ out, const float2* __restrict__ T, int64_t outer,
                      int Lin, int Lout, int64_t inner) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = outer * Lout * inner;
    if (e >= total) return;
    const int64_t i = e % inner;
    const int j = (int)((e / inner) % Lout);
    const int64_t o = e / (inner * Lout);
    float re = 0.f, im = 0.f;
    const float2* t = T + (int64_t)j * Lin;
    for (int q = 0; q < Lin; ++q) {
        const int64_t ii = (o * Lin + q) * inner + i;
        const float2 w = t[q];
        if (CIN) {
            const float2 x = reinterpret_cast<const float2*>(in)[ii];
            re += w.x * x.x - w.y * x.y;
            im += w.x * x.y + w.y * x.x;
        } else {
            const float x = reinterpret_cast<const float*>(in)[ii];
            re += w.x * x;
            im += w.y * x;
        }
    }
    if (COUT) reinterpret_cast<float2*>(out)[e] = make_float2(re, im);
    else reinterpret_cast<float*>(out)[e] = re;
}

// G[b][o][k] = sum_c R[k][o][c] V[b][c][k]; R as BF16 (or FP32) real/imag planes
template <class TR>
__global__ void k_mix(const TR* __restrict__ Rr, const TR* __restrict__ Ri, const float2* __restrict__ V,
                      float2* __restrict__ G, int B, int C, int64_t K, int conj_adj) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * C * K) return;
    const int64_t k = e % K;
    const int o = (int)((e / K) % C);
    const int b = (int)(e / (K * C));
    float re = 0.f, im = 0.f;
    for (int c = 0; c < C; ++c) {
        // forward: R[k][o][c]; adjoint (conj_adj): conj(R[k][c][o])
        const int64_t ri = conj_adj ? (k * C + c) * C + o : (k * C + o) * C + c;
        const float ar = (float)Rr[ri], ai = conj_adj ? -(float)Ri[ri] : (float)Ri[ri];
        const float2 x = V[((int64_t)b * C + c) * K + k];
        re += ar * x.x - ai * x.y;
        im += ar * x.y + ai * x.x;
    }
    G[e] = make_float2(re, im);
}

// dR[k][o][c] += sum_b dG[b][o][k] conj(V[b][c][k])  (real and imaginary planes)
__global__ void k_mix_grad(const float2* __restrict__ dG, const float2* __restrict__ V, float* dRr, float* dRi, int B,
                           int C, int64_t K) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * C * C) return;
    const int c = (int)(e % C);
    const int o = (int)((e / C) % C);
    const int64_t k = e / ((int64_t)C * C);
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
        const float2 g = dG[((int64_t)b * C + o) * K + k];
        const float2 x = V[((int64_t)b * C + c) * K + k];
        re += g.x * x.x + g.y * x.y;
        im += g.y * x.x - g.x * x.y;
    }
    dRr[e] += re;
    dRi[e] += im;
}

// lift: v0[b][c][p] = Wl[c] u[b][p] + bl[c]
__global__ void k_lift(const float* u, const float* Wl, const float* bl, float* v0, int B, int C, int64_t np3) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * C * np3) return;
    const int64_t p = e % np3;
    const int c = (int)((e / np3) % C);
    const int b = (int)(e / (np3 * C));
    v0[e] = Wl[c] * u[(int64_t)b * np3 + p] + bl[c];
}

// pointwise layer: z = s + W v + b, vout = GELU(z) (or z for the last layer); one thread per point
constexpr int MAXC = 64;
constexpr int SNO_MAX_JUDGE = 4096;   // most judge targets per photo_solve
__global__ void k_point(const float* s, const float* v, const float* W, const float* bias, float* z, float* vout,
                        int B, int C, int64_t np3, int act) {
    __shared__ float Ws[MAXC * MAXC], bs[MAXC];
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) Ws[i] = W[i];
    for (int i = threadIdx.x; i < C; i += blockDim.x) bs[i] = bias[i];
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * np3) return;
    const int64_t p = e % np3, b = e / np3;
    float x[MAXC];
    for (int c = 0; c < C; ++c) x[c] = v[(b * C + c) * np3 + p];
    for (int o = 0; o < C; ++o) {
        float a = bs[o] + s[(b * C + o) * np3 + p];
        for (int c = 0; c < C; ++c) a += Ws[o * C + c] * x[c];
        z[(b * C + o) * np3 + p] = a;
        vout[(b * C + o) * np3 + p] = act ? gelu_f(a) : a;
    }
}

// projection: y = Q2 . GELU(Q1 v + q1) + q2
__global__ void k_proj(const float* v, const float* Q1, const float* q1, const float* Q2, const float* q2, float* y,
                       int B, int C, int P, int64_t np3) {
    __shared__ float Qs[MAXC * MAXC * 2], qs[2 * MAXC], q2s[2 * MAXC];
    for (int i = threadIdx.x; i < P * C; i += blockDim.x) Qs[i] = Q1[i];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        qs[i] = q1[i];
        q2s[i] = Q2[i];
    }
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * np3) return;
    const int64_t p = e % np3, b = e / np3;
    float x[MAXC];
    for (int c = 0; c < C; ++c) x[c] = v[(b * C + c) * np3 + p];
    float out = q2[0];
    for (int o = 0; o < P; ++o) {
        float a = qs[o];
        for (int c = 0; c < C; ++c) a += Qs[o * C + c] * x[c];
        out += q2s[o] * gelu_f(a);
    }
    y[e] = out;
}

// loss and dL/dy: mean squared error; dy = 2 (y - t) / (B np3)
__global__ void k_loss(const float* y, const float* t, float* dy, int64_t N, double* loss) {
    __shared__ double red[256];
    double acc = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[e] - t[e];
        acc += (double)d * d;
        dy[e] = 2.0f * d / (float)N;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)N);
}

// projection backward, per point: a = Q1 v + q1, h = GELU(a), da = dy Q2 .* GELU'(a),
// dv = Q1^T da (h and da stored for the weight gradients)
__global__ void k_proj_bwd(const float* v, const float* dy, const float* Q1, const float* q1, const float* Q2,
                           float* h, float* da, float* dv, int B, int C, int P, int64_t np3) {
    __shared__ float Qs[MAXC * MAXC * 2], qs[2 * MAXC], q2s[2 * MAXC];
    for (int i = threadIdx.x; i < P * C; i += blockDim.x) Qs[i] = Q1[i];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        qs[i] = q1[i];
        q2s[i] = Q2[i];
    }
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * np3) return;
    const int64_t p = e % np3, b = e / np3;
    float x[MAXC], g[MAXC];
    for (int c = 0; c < C; ++c) {
        x[c] = v[(b * C + c) * np3 + p];
        g[c] = 0.f;
    }
    const float d = dy[e];
    for (int o = 0; o < P; ++o) {
        float a = qs[o];
        for (int c = 0; c < C; ++c) a += Qs[o * C + c] * x[c];
        h[(b * P + o) * np3 + p] = gelu_f(a);
        const float dd = d * q2s[o] * gelu_d(a);
        da[(b * P + o) * np3 + p] = dd;
        for (int c = 0; c < C; ++c) g[c] += Qs[o * C + c] * dd;
    }
    for (int c = 0; c < C; ++c) dv[(b * C + c) * np3 + p] = g[c];
}

// pointwise layer backward, per point: dz = dvout .* GELU'(z) (or dvout), dvin = W^T dz
// (in place: dvout and dvin may alias; each thread owns its point)
__global__ void k_point_bwd(const float* dvout, const float* z, const float* W, float* dz, float* dvin, int B, int C,
                            int64_t np3, int act) {
    __shared__ float Ws[MAXC * MAXC];
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) Ws[i] = W[i];
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * np3) return;
    const int64_t p = e % np3, b = e / np3;
    float d[MAXC];
    for (int o = 0; o < C; ++o) {
        const int64_t ii = (b * C + o) * np3 + p;
        const float g = dvout[ii];
        d[o] = act ? g * gelu_d(z[ii]) : g;
        dz[ii] = d[o];
    }
    for (int c = 0; c < C; ++c) {
        float a = 0.f;
        for (int o = 0; o < C; ++o) a += Ws[o * C + c] * d[o];
        dvin[(b * C + c) * np3 + p] = a;
    }
}

// weight gradient as a reduction GEMM: out[a][c] += sum over points (b, p) of
// A[b][a][p] * Bm[b][c][p] (A: Ca rows, Bm: Cb rows, both [B][rows][np3], Ca, Cb <= 128).
// Block (x, y) takes chunk x of the points and outputs y*OS_OUT .. y*OS_OUT + OS_OUT - 1,
// stages 32 points at a time, accumulates its partial in registers (8 outputs per
// thread of 256) and adds it to the gradient atomically.
constexpr int OS_CHUNK = 2048, OS_OUT = 2048;
__global__ void __launch_bounds__(256) k_outer_sum(const float* A, const float* Bm, float* out, int Ca, int Cb, int B,
                                                   int64_t np3) {
    __shared__ float As[2 * MAXC][33], Bs[2 * MAXC][33];
    const int64_t N = (int64_t)B * np3;
    const int64_t e0 = (int64_t)blockIdx.x * OS_CHUNK;
    const int nout = Ca * Cb;
    const int obase = blockIdx.y * OS_OUT;
    float acc[8] = {};
    for (int64_t s0 = e0; s0 < e0 + OS_CHUNK && s0 < N; s0 += 32) {
        __syncthreads();
        for (int i = threadIdx.x; i < (Ca + Cb) * 32; i += blockDim.x) {
            const int r = i / 32, k = i % 32;
            const int64_t e = s0 + k;
            float val = 0.f;
            if (e < N) {
                const int64_t b = e / np3, p = e % np3;
                val = r < Ca ? A[(b * Ca + r) * np3 + p] : Bm[(b * Cb + (r - Ca)) * np3 + p];
            }
            if (r < Ca) As[r][k] = val;
            else Bs[r - Ca][k] = val;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int o = obase + threadIdx.x + t * 256;
            if (o < nout) {
                const int a = o / Cb, c = o % Cb;
                float s = 0.f;
#pragma unroll 8
                for (int k = 0; k < 32; ++k) s += As[a][k] * Bs[c][k];
                acc[t] += s;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int o = obase + threadIdx.x + t * 256;
        if (o < nout) atomicAdd(&out[o], acc[t]);
    }
}

// row sums out[r] += sum over (b, p) of A[b][r][p]
__global__ void k_row_sum(const float* A, float* out, int R, int B, int64_t np3) {
    __shared__ float s1[256];
    const int r = blockIdx.y;
    float a = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)B * np3;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % np3, b = e / np3;
        a += A[(b * R + r) * np3 + p];
    }
    s1[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s1[threadIdx.x] += s1[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&out[r], s1[0]);
}

__global__ void k_add(float* a, const float* b, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) a[e] += b[e];
}

// lift backward: gWl[c] += sum dv0 * u, gbl[c] += sum dv0
__global__ void k_lift_bwd(const float* dv0, const float* u, float* gWl, float* gbl, int B, int C, int64_t np3) {
    __shared__ float s1[256], s2[256];
    const int c = blockIdx.y;
    float a = 0.f, bsum = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)B * np3;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % np3, b = e / np3;
        const float g = dv0[(b * C + c) * np3 + p];
        a += g * u[e];
        bsum += g;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = bsum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&gWl[c], s1[0]);
        atomicAdd(&gbl[c], s2[0]);
    }
}

__global__ void k_adam(float* th, const float* g, float* mo, float* ve, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float m = b1 * mo[e] + (1.f - b1) * gi;
    const float v = b2 * ve[e] + (1.f - b2) * gi * gi;
    mo[e] = m;
    ve[e] = v;
    th[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_to_bf16(const float* a, __nv_bfloat16* b, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = __float2bfloat16_rn(a[e]);
}

// ---- passes ---------------------------------------------------------------------------------
static float* act(DevBuf& b, int64_t i, int64_t per) { return ptr<float>(b) + i * per; }

// spectral convolution s = SpecConv(v) for layer l (B samples); cz/cy/cx/g/gx/gy scratch
static int spec_forward(SnoModel& M, int l, const float* v, float* s, int B) {
    const int n = M.n, m = M.m, C = M.C;
    const int64_t BC = (int64_t)B * C;
    const float2* T = ptr<float2>(M.tabs);
    cudaStream_t st = M.st;
    float2* cz = ptr<float2>(M.cz);
    float2* cy = ptr<float2>(M.cy);
    float2* cx = ptr<float2>(M.cx);
    float2* g = ptr<float2>(M.g);
    float2* gx = ptr<float2>(M.gx);
    float2* gy = ptr<float2>(M.gy);
    int64_t tot;
    tot = BC * n * n * m;   // z: [BC*n*n][n] -> [BC*n*n][m]
    k_dft<false, true><<<nbs(tot, 256), 256, 0, st>>>(v, cz, T + M.tzf, BC * n * n, n, m, 1);
    KF_LAUNCH();
    tot = BC * n * (2 * m) * m;   // y: [BC*n][n][m] -> [BC*n][2m][m]
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(cz, cy, T + M.tyf, BC * n, n, 2 * m, m);
    KF_LAUNCH();
    tot = BC * (2 * m) * (2 * m) * m;   // x: [BC][n][2m*m] -> [BC][2m][2m*m]
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(cy, cx, T + M.tyf, BC, n, 2 * m, (int64_t)2 * m * m);
    KF_LAUNCH();
    tot = BC * M.K;
    if (M.bf16)
        k_mix<__nv_bfloat16><<<nbs(tot, 256), 256, 0, st>>>(
            ptr<__nv_bfloat16>(M.rbf) + (int64_t)l * 2 * M.K * C * C,
            ptr<__nv_bfloat16>(M.rbf) + ((int64_t)l * 2 + 1) * M.K * C * C, cx, g, B, C, M.K, 0);
    else
        k_mix<float><<<nbs(tot, 256), 256, 0, st>>>(ptr<float>(M.theta) + M.off[o_rr(l)],
                                                    ptr<float>(M.theta) + M.off[o_ri(l)], cx, g, B, C, M.K, 0);
    KF_LAUNCH();
    tot = BC * n * (2 * m) * m;   // inverse x: [BC][2m][2m*m] -> [BC][n][2m*m]
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(g, gx, T + M.txi, BC, 2 * m, n, (int64_t)2 * m * m);
    KF_LAUNCH();
    tot = BC * n * n * m;   // inverse y: [BC*n][2m][m] -> [BC*n][n][m]
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(gx, gy, T + M.txi, BC * n, 2 * m, n, m);
    KF_LAUNCH();
    tot = BC * n * n * n;   // inverse z (real part, weights w/n^3): [BC*n*n][m] -> [BC*n*n][n]
    k_dft<true, false><<<nbs(tot, 256), 256, 0, st>>>(gy, s, T + M.tzi, BC * n * n, m, n, 1);
    KF_LAUNCH();
    return KIFMM_OK;
}

static int forward(SnoModel& M, const float* u, float* y, int B) {
    const int64_t per = (int64_t)B * M.C * M.np3;
    cudaStream_t st = M.st;
    const float* th = ptr<float>(M.theta);
    k_lift<<<nbs(per, 256), 256, 0, st>>>(u, th + M.off[O_WL], th + M.off[O_BL], act(M.v, 0, per), B, M.C, M.np3);
    KF_LAUNCH();
    for (int l = 0; l < M.L; ++l) {
        KF_TRY(spec_forward(M, l, act(M.v, l, per), ptr<float>(M.s), B));
        k_point<<<nbs((int64_t)B * M.np3, 128), 128, 0, st>>>(ptr<float>(M.s), act(M.v, l, per), th + M.off[o_w(l)],
                                                              th + M.off[o_b(l)], act(M.z, l, per),
                                                              act(M.v, l + 1, per), B, M.C, M.np3, l < M.L - 1);
        KF_LAUNCH();
    }
    const int q = o_q1(M);
    k_proj<<<nbs((int64_t)B * M.np3, 128), 128, 0, st>>>(act(M.v, M.L, per), th + M.off[q], th + M.off[q + 1],
                                                         th + M.off[q + 2], th + M.off[q + 3], y, B, M.C, M.P,
                                                         M.np3);
    KF_LAUNCH();
    return KIFMM_OK;
}

// adjoint of SpecConv for layer l: dvin += SpecConv^T(dz); dR accumulated
static int spec_backward(SnoModel& M, int l, const float* dz, const float* v, float* dvin, int B) {
    const int n = M.n, m = M.m, C = M.C;
    const int64_t BC = (int64_t)B * C;
    const float2* T = ptr<float2>(M.tabs);
    cudaStream_t st = M.st;
    float2* cz = ptr<float2>(M.cz);
    float2* cy = ptr<float2>(M.cy);
    float2* cx = ptr<float2>(M.cx);
    float2* g = ptr<float2>(M.g);
    float2* gx = ptr<float2>(M.gx);
    float2* gy = ptr<float2>(M.gy);
    int64_t tot;
    // recompute the forward spectrum V of v (cx) for the weight gradient
    tot = BC * n * n * m;
    k_dft<false, true><<<nbs(tot, 256), 256, 0, st>>>(v, cz, T + M.tzf, BC * n * n, n, m, 1);
    KF_LAUNCH();
    tot = BC * n * (2 * m) * m;
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(cz, cy, T + M.tyf, BC * n, n, 2 * m, m);
    KF_LAUNCH();
    tot = BC * (2 * m) * (2 * m) * m;
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(cy, cx, T + M.tyf, BC, n, 2 * m, (int64_t)2 * m * m);
    KF_LAUNCH();
    // adjoint of the inverse transforms: dGy = (w/n^3) DFT_z(dz), dGx = DFT_y, dG = DFT_x
    tot = BC * n * n * m;
    k_dft<false, true><<<nbs(tot, 256), 256, 0, st>>>(dz, gy, T + M.tzb, BC * n * n, n, m, 1);
    KF_LAUNCH();
    tot = BC * n * (2 * m) * m;
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(gy, gx, T + M.tyf, BC * n, n, 2 * m, m);
    KF_LAUNCH();
    tot = BC * (2 * m) * (2 * m) * m;
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(gx, g, T + M.tyf, BC, n, 2 * m, (int64_t)2 * m * m);
    KF_LAUNCH();
    // weight gradient and the adjoint of the mixing: dV = R^H dG (into cy's storage)
    float* gRr = ptr<float>(M.grad) + M.off[o_rr(l)];
    float* gRi = ptr<float>(M.grad) + M.off[o_ri(l)];
    k_mix_grad<<<nbs(M.K * C * C, 256), 256, 0, st>>>(g, cx, gRr, gRi, B, C, M.K);
    KF_LAUNCH();
    float2* dV = cx;   // V no longer needed
    tot = BC * M.K;
    float2* gtmp = cy;
    if (M.bf16)
        k_mix<__nv_bfloat16><<<nbs(tot, 256), 256, 0, st>>>(
            ptr<__nv_bfloat16>(M.rbf) + (int64_t)l * 2 * M.K * C * C,
            ptr<__nv_bfloat16>(M.rbf) + ((int64_t)l * 2 + 1) * M.K * C * C, g, gtmp, B, C, M.K, 1);
    else
        k_mix<float><<<nbs(tot, 256), 256, 0, st>>>(ptr<float>(M.theta) + M.off[o_rr(l)],
                                                    ptr<float>(M.theta) + M.off[o_ri(l)], g, gtmp, B, C, M.K, 1);
    KF_LAUNCH();
    (void)dV;
    // adjoint of the forward transforms: inverse-type x, y, then z (real part, unit weights)
    tot = BC * n * (2 * m) * m;
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(gtmp, gx, T + M.txi, BC, 2 * m, n, (int64_t)2 * m * m);
    KF_LAUNCH();
    tot = BC * n * n * m;
    k_dft<true, true><<<nbs(tot, 256), 256, 0, st>>>(gx, gy, T + M.txi, BC * n, 2 * m, n, m);
    KF_LAUNCH();
    tot = BC * n * n * n;
    k_dft<true, false><<<nbs(tot, 256), 256, 0, st>>>(gy, ptr<float>(M.s), T + M.tzr, BC * n * n, m, n, 1);
    KF_LAUNCH();
    k_add<<<nbs(tot, 256), 256, 0, st>>>(dvin, ptr<float>(M.s), tot);
    KF_LAUNCH();
    return KIFMM_OK;
}

// loss, gradients (into M.grad, zeroed first)
static int outer_sum(SnoModel& M, const float* A, const float* Bm, float* out, int Ca, int Cb, int B) {
    const int64_t N = (int64_t)B * M.np3;
    k_outer_sum<<<dim3(nbs(N, OS_CHUNK), nbs((int64_t)Ca * Cb, OS_OUT)), 256, 0, M.st>>>(A, Bm, out, Ca, Cb, B,
                                                                                          M.np3);
    KF_LAUNCH();
    return KIFMM_OK;
}
static int row_sum(SnoModel& M, const float* A, float* out, int R, int B) {
    k_row_sum<<<dim3(256, R), 256, 0, M.st>>>(A, out, R, B, M.np3);
    KF_LAUNCH();
    return KIFMM_OK;
}

static int loss_grad(SnoModel& M, const float* u, const float* t, int B, double* loss_host) {
    cudaStream_t st = M.st;
    const int64_t per = (int64_t)B * M.C * M.np3, N = (int64_t)B * M.np3;
    float* gr = ptr<float>(M.grad);
    const float* th = ptr<float>(M.theta);
    KF_CUDA(cudaMemsetAsync(gr, 0, M.nparam * 4, st));
    KF_CUDA(cudaMemsetAsync(M.loss.p, 0, 8, st));
    float* y = ptr<float>(M.s) + per;   // the s buffer holds per + 3 N floats at least
    float* dy = y + N;
    KF_TRY(forward(M, u, y, B));
    k_loss<<<1024, 256, 0, st>>>(y, t, dy, N, ptr<double>(M.loss));
    KF_LAUNCH();
    const int q = o_q1(M);
    float* hbuf = ptr<float>(M.ph);
    float* dabuf = ptr<float>(M.pda);
    k_proj_bwd<<<nbs(N, 128), 128, 0, st>>>(act(M.v, M.L, per), dy, th + M.off[q], th + M.off[q + 1], th + M.off[q + 2],
                                            hbuf, dabuf, ptr<float>(M.dv), B, M.C, M.P, M.np3);
    KF_LAUNCH();
    KF_TRY(outer_sum(M, dabuf, act(M.v, M.L, per), gr + M.off[q], M.P, M.C, B));   // Q1
    KF_TRY(row_sum(M, dabuf, gr + M.off[q + 1], M.P, B));                          // q1
    KF_TRY(outer_sum(M, dy, hbuf, gr + M.off[q + 2], 1, M.P, B));                  // Q2
    KF_TRY(row_sum(M, dy, gr + M.off[q + 3], 1, B));                               // q2
    for (int l = M.L - 1; l >= 0; --l) {
        // dv holds dL/dv_{l+1}; dz <- it times GELU'(z_l); dv <- W^T dz + SpecConv^T dz
        k_point_bwd<<<nbs(N, 128), 128, 0, st>>>(ptr<float>(M.dv), act(M.z, l, per), th + M.off[o_w(l)],
                                                 ptr<float>(M.dz), ptr<float>(M.dv), B, M.C, M.np3, l < M.L - 1);
        KF_LAUNCH();
        KF_TRY(outer_sum(M, ptr<float>(M.dz), act(M.v, l, per), gr + M.off[o_w(l)], M.C, M.C, B));
        KF_TRY(row_sum(M, ptr<float>(M.dz), gr + M.off[o_b(l)], M.C, B));
        KF_TRY(spec_backward(M, l, ptr<float>(M.dz), act(M.v, l, per), ptr<float>(M.dv), B));
    }
    k_lift_bwd<<<dim3(256, M.C), 256, 0, st>>>(ptr<float>(M.dv), u, gr + M.off[O_WL], gr + M.off[O_BL], B, M.C,
                                               M.np3);
    KF_LAUNCH();
    if (loss_host) {
        KF_CUDA(cudaMemcpyAsync(loss_host, M.loss.p, 8, cudaMemcpyDeviceToHost, st));
        KF_CUDA(cudaStreamSynchronize(st));
    }
    return KIFMM_OK;
}

static int refresh_bf16(SnoModel& M) {
    const int64_t KC = M.K * M.C * M.C;
    for (int l = 0; l < M.L; ++l) {
        k_to_bf16<<<nbs(KC, 256), 256, 0, M.st>>>(ptr<float>(M.theta) + M.off[o_rr(l)],
                                                  ptr<__nv_bfloat16>(M.rbf) + (int64_t)l * 2 * KC, KC);
        KF_LAUNCH();
        k_to_bf16<<<nbs(KC, 256), 256, 0, M.st>>>(ptr<float>(M.theta) + M.off[o_ri(l)],
                                                  ptr<__nv_bfloat16>(M.rbf) + ((int64_t)l * 2 + 1) * KC, KC);
        KF_LAUNCH();
    }
    return KIFMM_OK;
}

// ---- judge: direct sum at sampled targets (FP32, absolute coordinates) ------------------------
__global__ void k_judge(const double* pts, const double* q, const int32_t* targets, int k, int64_t n, KParams kp,
                        const double* sigma, const double* Isort, double C, const int32_t* perm, double* ref,
                        int32_t* orig) {
    const int t = blockIdx.x;
    if (t >= k) return;
    const int64_t i = targets[t];
    const float xi = (float)pts[3 * i], yi = (float)pts[3 * i + 1], zi = (float)pts[3 * i + 2];
    __shared__ double red[256];
    double acc = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        if (j == i) continue;
        const float dx = xi - (float)pts[3 * j], dy = yi - (float)pts[3 * j + 1], dz = zi - (float)pts[3 * j + 2];
        acc += (double)kern_f32(dx * dx + dy * dy + dz * dz, kp) * q[j];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ref[t] = C * (red[0] + sigma[i] * Isort[i]);
        orig[t] = perm[i];
    }
}

__global__ void k_log1p_in(const double* I, float* u, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) u[e] = (float)log1p(fmax(I[e], 0.0));
}
__global__ void k_expm1_out(const float* y, double* S, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) S[e] = expm1((double)y[e]);
}
__global__ void k_judge_err(const double* S, const double* ref, const int32_t* orig, int k, double* out) {
    __shared__ double a[256], b[256];
    double num = 0, den = 0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const double d = S[orig[t]] - ref[t];
        num += d * d;
        den += ref[t] * ref[t];
    }
    a[threadIdx.x] = num;
    b[threadIdx.x] = den;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(a[0] / fmax(b[0], 1e-300));
}

}  // namespace kifmm

using namespace kifmm;

struct sno_model_s {
    SnoModel m;
};

extern "C" {

int sno_create(sno_model_t* out, int n, int width, int modes, int layers, int proj_width, int max_batch,
               void* stream) {
    set_error("");
    if (!out || n < 4 || width < 1 || width > MAXC || modes < 1 || 2 * modes > n || layers < 1 ||
        proj_width < 1 || proj_width > 2 * MAXC || max_batch < 1) {
        set_error("sno_create: invalid dimensions");
        return KIFMM_ERR_ARG;
    }
    *out = nullptr;
    sno_model_s* h = new (std::nothrow) sno_model_s();
    if (!h) return KIFMM_ERR_OOM;
    SnoModel& M = h->m;
    M.n = n;
    M.C = width;
    M.m = modes;
    M.L = layers;
    M.P = proj_width;
    M.maxB = max_batch;
    M.st = (cudaStream_t)stream;
    M.K = (int64_t)(2 * modes) * (2 * modes) * modes;
    M.np3 = (int64_t)n * n * n;
    sno_layout(M);
    auto fail = [&](int rc) {
        sno_destroy(h);
        return rc;
    };
    const int64_t per = (int64_t)max_batch * width * M.np3;
    const int64_t BC = (int64_t)max_batch * width;
    int rc = KIFMM_OK;
    for (auto* pr : {&M.theta, &M.grad, &M.adam_m, &M.adam_v}) {
        rc = dev_alloc(*pr, M.nparam * 4);
        if (rc) return fail(rc);
        if (cudaMemsetAsync(pr->p, 0, M.nparam * 4, M.st) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    }
    if ((rc = dev_alloc(M.rbf, (size_t)layers * 2 * M.K * width * width * 2))) return fail(rc);
    M.tzf = 0;
    M.tyf = M.tzf + (int64_t)modes * n;
    M.tzb = M.tyf + (int64_t)2 * modes * n;
    M.txi = M.tzb + (int64_t)modes * n;
    M.tzi = M.txi + (int64_t)n * 2 * modes;
    M.tzr = M.tzi + (int64_t)n * modes;
    if ((rc = dev_alloc(M.tabs, (M.tzr + (int64_t)n * modes) * sizeof(float2)))) return fail(rc);
    k_tables<<<nbs(2 * modes * n, 128), 128, 0, M.st>>>(n, modes, ptr<float2>(M.tabs), M.tzf, M.tyf, M.tzb, M.txi,
                                                          M.tzi, M.tzr);
    if (cudaGetLastError() != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    if ((rc = dev_alloc(M.v, (size_t)(layers + 1) * per * 4))) return fail(rc);
    if ((rc = dev_alloc(M.z, (size_t)layers * per * 4))) return fail(rc);
    if ((rc = dev_alloc(M.s, (size_t)std::max<int64_t>(per, 3 * (int64_t)max_batch * M.np3) * 4 + per * 4)))
        return fail(rc);
    if ((rc = dev_alloc(M.dv, (size_t)per * 4))) return fail(rc);
    if ((rc = dev_alloc(M.dz, (size_t)per * 4))) return fail(rc);
    if ((rc = dev_alloc(M.cz, (size_t)BC * n * n * modes * 8))) return fail(rc);
    if ((rc = dev_alloc(M.cy, (size_t)std::max<int64_t>(BC * n * 2 * modes * modes, BC * M.K) * 8))) return fail(rc);
    if ((rc = dev_alloc(M.cx, (size_t)BC * M.K * 8))) return fail(rc);
    if ((rc = dev_alloc(M.g, (size_t)BC * M.K * 8))) return fail(rc);
    if ((rc = dev_alloc(M.gx, (size_t)BC * n * 2 * modes * modes * 8))) return fail(rc);
    if ((rc = dev_alloc(M.gy, (size_t)BC * n * n * modes * 8))) return fail(rc);
    if ((rc = dev_alloc(M.loss, 16))) return fail(rc);
    if ((rc = dev_alloc(M.ph, (size_t)max_batch * proj_width * M.np3 * 4))) return fail(rc);
    if ((rc = dev_alloc(M.pda, (size_t)max_batch * proj_width * M.np3 * 4))) return fail(rc);
    if ((rc = dev_alloc(M.jt, SNO_MAX_JUDGE * 4))) return fail(rc);
    if ((rc = dev_alloc(M.jref, SNO_MAX_JUDGE * 8))) return fail(rc);
    if ((rc = dev_alloc(M.jorig, SNO_MAX_JUDGE * 4))) return fail(rc);
    if ((rc = dev_alloc(M.jerr, 8))) return fail(rc);
    if (cudaStreamSynchronize(M.st) != cudaSuccess) return fail(KIFMM_ERR_CUDA);
    *out = h;
    return KIFMM_OK;
}

void sno_destroy(sno_model_t h) {
    if (!h) return;
    SnoModel& M = h->m;
    if (M.st) cudaStreamSynchronize(M.st);
    for (DevBuf* b : {&M.theta, &M.grad, &M.adam_m, &M.adam_v, &M.rbf, &M.tabs, &M.v, &M.z, &M.s, &M.cz, &M.cy,
                      &M.cx, &M.g, &M.gx, &M.gy, &M.dv, &M.dz, &M.loss, &M.ph, &M.pda, &M.jt, &M.jref,
                      &M.jorig, &M.jerr})
        dev_free(*b);
    delete h;
}

int64_t sno_num_params(sno_model_t h) { return h ? h->m.nparam : -1; }

int sno_set_params(sno_model_t h, const float* theta_host) {
    if (!h || !theta_host) {
        set_error("sno_set_params: invalid argument");
        return KIFMM_ERR_ARG;
    }
    SnoModel& M = h->m;
    KF_CUDA(cudaMemcpyAsync(M.theta.p, theta_host, M.nparam * 4, cudaMemcpyHostToDevice, M.st));
    KF_CUDA(cudaMemsetAsync(M.adam_m.p, 0, M.nparam * 4, M.st));
    KF_CUDA(cudaMemsetAsync(M.adam_v.p, 0, M.nparam * 4, M.st));
    M.steps = 0;
    KF_TRY(refresh_bf16(M));
    KF_CUDA(cudaStreamSynchronize(M.st));
    return KIFMM_OK;
}

int sno_get_params(sno_model_t h, float* theta_host) {
    if (!h || !theta_host) return KIFMM_ERR_ARG;
    KF_CUDA(cudaMemcpyAsync(theta_host, h->m.theta.p, h->m.nparam * 4, cudaMemcpyDeviceToHost, h->m.st));
    KF_CUDA(cudaStreamSynchronize(h->m.st));
    return KIFMM_OK;
}

int sno_get_grads(sno_model_t h, float* grad_host) {
    if (!h || !grad_host) return KIFMM_ERR_ARG;
    KF_CUDA(cudaMemcpyAsync(grad_host, h->m.grad.p, h->m.nparam * 4, cudaMemcpyDeviceToHost, h->m.st));
    KF_CUDA(cudaStreamSynchronize(h->m.st));
    return KIFMM_OK;
}

// file: "SNO1", int32 n, width, modes, layers, proj_width, int64 parameter count, FP32 parameters
int sno_save(sno_model_t h, const char* path) {
    set_error("");
    if (!h || !path) return KIFMM_ERR_ARG;
    SnoModel& M = h->m;
    std::vector<float> th(M.nparam);
    KF_CUDA(cudaMemcpyAsync(th.data(), M.theta.p, M.nparam * 4, cudaMemcpyDeviceToHost, M.st));
    KF_CUDA(cudaStreamSynchronize(M.st));
    FILE* fp = fopen(path, "wb");
    if (!fp) {
        set_error("sno_save: cannot open the file");
        return KIFMM_ERR_ARG;
    }
    const int32_t hdr[6] = {0x314f4e53, M.n, M.C, M.m, M.L, M.P};
    bool ok = fwrite(hdr, 4, 6, fp) == 6 && fwrite(&M.nparam, 8, 1, fp) == 1 &&
              fwrite(th.data(), 4, M.nparam, fp) == (size_t)M.nparam;
    ok = (fclose(fp) == 0) && ok;
    if (!ok) {
        set_error("sno_save: write failed");
        return KIFMM_ERR_ARG;
    }
    return KIFMM_OK;
}

int sno_load(sno_model_t h, const char* path) {
    set_error("");
    if (!h || !path) return KIFMM_ERR_ARG;
    SnoModel& M = h->m;
    FILE* fp = fopen(path, "rb");
    if (!fp) {
        set_error("sno_load: cannot open the file");
        return KIFMM_ERR_ARG;
    }
    int32_t hdr[6] = {0};
    int64_t np = -1;
    std::vector<float> th(M.nparam);
    bool ok = fread(hdr, 4, 6, fp) == 6 && fread(&np, 8, 1, fp) == 1;
    ok = ok && hdr[0] == 0x314f4e53 && hdr[1] == M.n && hdr[2] == M.C && hdr[3] == M.m && hdr[4] == M.L &&
         hdr[5] == M.P && np == M.nparam;
    ok = ok && fread(th.data(), 4, M.nparam, fp) == (size_t)M.nparam;
    fclose(fp);
    if (!ok) {
        set_error("sno_load: not a parameter file of this model's shape");
        return KIFMM_ERR_ARG;
    }
    return sno_set_params(h, th.data());
}

int sno_set_bf16(sno_model_t h, int on) {
    if (!h) return KIFMM_ERR_ARG;
    h->m.bf16 = on ? 1 : 0;
    return refresh_bf16(h->m);
}

int sno_forward(sno_model_t h, const float* u_dev, float* y_dev, int batch) {
    if (!h || !u_dev || !y_dev || batch < 1 || batch > h->m.maxB) {
        set_error("sno_forward: invalid argument");
        return KIFMM_ERR_ARG;
    }
    return forward(h->m, u_dev, y_dev, batch);
}

int sno_loss_grad(sno_model_t h, const float* u_dev, const float* t_dev, int batch, double* loss) {
    if (!h || !u_dev || !t_dev || batch < 1 || batch > h->m.maxB) {
        set_error("sno_loss_grad: invalid argument");
        return KIFMM_ERR_ARG;
    }
    return loss_grad(h->m, u_dev, t_dev, batch, loss);
}

int sno_adam_step(sno_model_t h, float lr, float beta1, float beta2, float eps) {
    if (!h) return KIFMM_ERR_ARG;
    SnoModel& M = h->m;
    M.steps += 1;
    const float c1 = 1.f - powf(beta1, (float)M.steps), c2 = 1.f - powf(beta2, (float)M.steps);
    k_adam<<<nbs(M.nparam, 256), 256, 0, M.st>>>(ptr<float>(M.theta), ptr<float>(M.grad), ptr<float>(M.adam_m),
                                                 ptr<float>(M.adam_v), M.nparam, lr, beta1, beta2, eps, c1, c2);
    KF_LAUNCH();
    return refresh_bf16(M);
}

int photo_solve(kifmm_plan_t plan, sno_model_t model, const double* I_dev, double* S_dev, double C, double tol,
                int k_samples, uint64_t seed, int* used_fallback, double* judged_err) {
    set_error("");
    if (!plan || !model || !I_dev || !S_dev || k_samples < 1 || k_samples > SNO_MAX_JUDGE) {
        set_error("photo_solve: invalid argument");
        return KIFMM_ERR_ARG;
    }
    Plan& p = *kifmm_plan_internal(plan);
    SnoModel& M = model->m;
    const int64_t n = p.tree.n;
    if (n != M.np3) {
        set_error("photo_solve: the plan's point count differs from the model's grid");
        return KIFMM_ERR_ARG;
    }
    cudaStream_t st = p.stream;
    cudaStream_t saved = M.st;
    M.st = st;
    // surrogate: u = log(1 + I) in the caller's (grid) order, y -> S = e^y - 1
    float* u = ptr<float>(M.dv);
    float* y = ptr<float>(M.dz);
    k_log1p_in<<<nbs(n, 256), 256, 0, st>>>(I_dev, u, n);
    KF_LAUNCH();
    int rc = forward(M, u, y, 1);
    M.st = saved;
    KF_TRY(rc);
    k_expm1_out<<<nbs(n, 256), 256, 0, st>>>(y, S_dev, n);
    KF_LAUNCH();
    // judge: direct sum at k sampled targets (sorted indices drawn with a fixed LCG)
    std::vector<int32_t> tg(k_samples);
    uint64_t sst = seed * 6364136223846793005ull + 1442695040888963407ull;
    for (int t = 0; t < k_samples; ++t) {
        sst = sst * 6364136223846793005ull + 1442695040888963407ull;
        tg[t] = (int32_t)((sst >> 33) % (uint64_t)n);
    }
    DevBuf &dt = M.jt, &dref = M.jref, &dorig = M.jorig, &derr = M.jerr;
    KF_CUDA(cudaMemcpyAsync(dt.p, tg.data(), k_samples * 4, cudaMemcpyHostToDevice, st));
    // weights q = I h^3 in sorted order (the evaluation's own scatter kernel path)
    KF_TRY(kifmm_scatter_weights(p, I_dev));
    k_judge<<<k_samples, 256, 0, st>>>(ptr<double>(p.pts), ptr<double>(p.q), ptr<int32_t>(dt), k_samples, n,
                                       make_kparams(p.a, p.b), ptr<double>(p.sigma), ptr<double>(p.Isort), C,
                                       ptr<int32_t>(p.tree.perm), ptr<double>(dref), ptr<int32_t>(dorig));
    KF_LAUNCH();
    k_judge_err<<<1, 256, 0, st>>>(S_dev, ptr<double>(dref), ptr<int32_t>(dorig), k_samples, ptr<double>(derr));
    KF_LAUNCH();
    double err = 0;
    KF_CUDA(cudaMemcpyAsync(&err, derr.p, 8, cudaMemcpyDeviceToHost, st));
    KF_CUDA(cudaStreamSynchronize(st));
    if (judged_err) *judged_err = err;
    const int fb = !(err <= tol);
    if (used_fallback) *used_fallback = fb;
    if (fb) KF_TRY(kifmm_eval(plan, I_dev, S_dev, KIFMM_F64, C));
    return KIFMM_OK;
}

}  // extern "C"
