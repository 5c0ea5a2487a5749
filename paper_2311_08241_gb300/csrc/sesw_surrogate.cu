// Learned surrogate of one baroclinic step: a message-passing network on the
// vertex-element graph of the uploaded mesh, trained and run with the kernels below.
//
// Network (hidden width 64, 3 layers; weights bfloat16, accumulation float; the six
// message layers take bfloat16 inputs and run on the tensor cores, sesw_tc.cu):
//   vertex inputs  x_v = [eta/s_eta, H0/s_H]
//   element inputs x_e = [U/s_U, R/s_R, f/s_f, H0_e/s_H]
//   h_v = tanh(x_v Wv0 + bv0),  h_e = tanh(x_e We0 + be0)
//   per layer: z_e = [h_e, L sum_k dphi_k/dx h_vk, L sum_k dphi_k/dy h_vk],  h_e += tanh(z_e We + be)
//              z_v = [h_v, area-weighted mean of h_e over the vertex's triangles], h_v += tanh(z_v Wv + bv)
//   o_e = h_e Weo + beo (4),  o_v = h_v Wvo + bvo (1)
// Outputs are the one-step increments <<U>> - U = s_oU o_e[0:2], U^M - U = s_oU o_e[2:4]
// and eta_bar - eta = s_oeta o_v. A step applies them with eta^{n+1} = eta^n - tau
// div <<U>> (so volume and Eq. 4.11 hold exactly) and accepts the step only when the
// exactly summed momentum equation of the step holds to a tolerance; otherwise the
// plain subcycle runs instead.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "sesw_internal.h"
#include "sesw_msg.cuh"

namespace sesw {

namespace {

constexpr int HC = 64;            // hidden width
constexpr int NL = 3;             // message-passing layers
constexpr int TILE_ROWS = 64;     // rows per block of the matrix kernels
constexpr int WG_ROWS = 32;       // rows per smem tile of the weight-gradient kernel
constexpr int NSCALE = 8;         // eta, H, U, R, f, L, out_U, out_eta

enum { S_ETA = 0, S_H, S_U, S_R, S_F, S_L, S_OU, S_OETA };

// ------------------------------------------------------------------------- matrices
//
// out[n][j] = sum_i X[n][i] * Wm(i, j) (+ bias[j]), optionally tanh, optionally + res[n][j],
// with Wm(i, j) = W[i * P + j] (forward, W is Kin x P) or W[j * Kin + i] (input gradient,
// W is P x Kin). Each block computes 64 rows; thread (rg, cg) computes rows 4 rg .. 4 rg + 3
// and columns cg + 16 j.
template <int PT>
__global__ void __launch_bounds__(256)
k_mm(int N, int Kin, int P, const float *__restrict__ X, const __nv_bfloat16 *__restrict__ W, int trans,
     const float *__restrict__ bias, int act, const float *__restrict__ res, float *__restrict__ Y)
{
    extern __shared__ float sm[];
    const int ldx = Kin + 1;
    float *Xs = sm;                              // [64][Kin + 1]
    float *Ws = sm + TILE_ROWS * ldx;            // [Kin][P]
    for (int t = threadIdx.x; t < Kin * P; t += blockDim.x) {
        const int i = t / P, j = t % P;
        const float w = __bfloat162float(trans ? W[(size_t)j * Kin + i] : W[(size_t)i * P + j]);
        Ws[i * P + j] = w;
    }
    const int n0 = blockIdx.x * TILE_ROWS;
    for (int t = threadIdx.x; t < TILE_ROWS * Kin; t += blockDim.x) {
        const int r = t / Kin, i = t % Kin;
        Xs[r * ldx + i] = (n0 + r < N) ? X[(size_t)(n0 + r) * Kin + i] : 0.0f;
    }
    __syncthreads();
    const int rg = threadIdx.x >> 4, cg = threadIdx.x & 15;
    float acc[4][PT];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int j = 0; j < PT; j++) acc[r][j] = 0.0f;
    for (int i = 0; i < Kin; i++) {
        float a[4], w[PT];
#pragma unroll
        for (int r = 0; r < 4; r++) a[r] = Xs[(rg * 4 + r) * ldx + i];
#pragma unroll
        for (int j = 0; j < PT; j++) {
            const int col = cg + 16 * j;
            w[j] = col < P ? Ws[i * P + col] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int j = 0; j < PT; j++) acc[r][j] = fmaf(a[r], w[j], acc[r][j]);
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int n = n0 + rg * 4 + r;
        if (n >= N) continue;
#pragma unroll
        for (int j = 0; j < PT; j++) {
            const int col = cg + 16 * j;
            if (col >= P) continue;
            float v = acc[r][j];
            if (bias) v += bias[col];
            if (act) v = tanhf(v);
            if (res) v += res[(size_t)n * P + col];
            Y[(size_t)n * P + col] = v;
        }
    }
}

// Weight gradient of the small layers (the input layers, K = 2 or 6 and C = 64; the output
// layers, K = 64 and C = 4 or 1; the message layers run on the tensor cores):
//   partial[b][i * C + c] = sum_{n in rows of block b} Z[n][i] dA[n][c],
//   partial[b][K * C + c] = sum_{n in rows of block b} dA[n][c].
// A chunk of WG_ROWS rows of Z and dA is staged in shared memory with coalesced loads; thread t
// owns outputs t, t + 256, ... of the K * C + C and adds the chunk's rows in order.
__global__ void __launch_bounds__(256)
k_wgrad_small(int N, int K, int C, const float *__restrict__ Z, const float *__restrict__ dA, int rows_per_block,
              float *__restrict__ partial)
{
    __shared__ float Zs[WG_ROWS * HC];
    __shared__ float Ds[WG_ROWS * HC];
    constexpr int MAXO = 2;                      // outputs per thread: (K * C + C) <= 512
    float acc[MAXO] = {0.0f, 0.0f};
    const int nout = K * C + C;
    const int nb = blockIdx.x * rows_per_block, ne = min(N, nb + rows_per_block);
    for (int t0 = nb; t0 < ne; t0 += WG_ROWS) {
        const int nr = min(WG_ROWS, ne - t0);
        __syncthreads();
        for (int t = threadIdx.x; t < nr * K; t += blockDim.x) Zs[t] = Z[(size_t)t0 * K + t];
        for (int t = threadIdx.x; t < nr * C; t += blockDim.x) Ds[t] = dA[(size_t)t0 * C + t];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXO; q++) {
            const int o = threadIdx.x + q * 256;
            if (o >= nout) continue;
            float a = acc[q];
            if (o < K * C) {
                const int i = o / C, c = o % C;
                for (int r = 0; r < nr; r++) a = fmaf(Zs[r * K + i], Ds[r * C + c], a);
            } else {
                const int c = o - K * C;
                for (int r = 0; r < nr; r++) a += Ds[r * C + c];
            }
            acc[q] = a;
        }
    }
    float *out = partial + (size_t)blockIdx.x * nout;
#pragma unroll
    for (int q = 0; q < MAXO; q++) {
        const int o = threadIdx.x + q * 256;
        if (o < nout) out[o] = acc[q];
    }
}

// Sum the partials of nb blocks in block order into gW (K*C) and gb (C).
__global__ void k_reduce_partials(const float *__restrict__ partial, int nb, int len, float *__restrict__ gW,
                                  float *__restrict__ gb, int KC)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < nb; b++) s += partial[(size_t)b * len + i];
        if (i < KC)
            gW[i] = s;
        else
            gb[i - KC] = s;
    }
}

// dA = dY * (1 - Y^2) (derivative of tanh at the stored output Y).
__global__ void k_tanh_bwd(size_t n, const float *__restrict__ dY, const float *__restrict__ Y, float *__restrict__ dA)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dA[i] = dY[i] * (1.0f - Y[i] * Y[i]);
}

// ------------------------------------------------------------------------- messages
// thread per (node, channel), 64 channels per node

// Z_e = [h_e, L sum_k gx_k h_vk, L sum_k gy_k h_vk], rebuilt for the backward pass (the forward
// pass forms it inside the tensor-core layer). The message-layer inputs are rounded to
// bfloat16 values: the tensor-core layers read them as BF16 operands.
__global__ void k_msg_elem(int E, const int4 *__restrict__ etri, const float4 *__restrict__ egrad, float L,
                           const float *__restrict__ he, const float *__restrict__ hv, float *__restrict__ Z)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)E * HC;
         t += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(t / HC), c = (int)(t % HC);
        const int4 v = etri[e];
        const float4 g = egrad[e];
        const float h0 = hv[(size_t)v.x * HC + c], h1 = hv[(size_t)v.y * HC + c], h2 = hv[(size_t)v.z * HC + c];
        const float2 m = msg_elem_grad(g, h0, h1, h2, L);
        float *z = Z + (size_t)e * 3 * HC;
        z[c] = bf16_value(he[t]);
        z[HC + c] = bf16_value(m.x);
        z[2 * HC + c] = bf16_value(m.y);
    }
}

// dh_e += dZ_e[:, 0:64]
__global__ void k_msg_elem_adj_e(int E, const float *__restrict__ dZ, float *__restrict__ dhe)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)E * HC;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t e = t / HC;
        dhe[t] += dZ[e * 3 * HC + t % HC];
    }
}

// dh_v += L sum_{(e,k) at v} (gx_k dZ_e[64 + c] + gy_k dZ_e[128 + c])
__global__ void k_msg_elem_adj_v(int V, const int *__restrict__ voff, const int *__restrict__ vinc,
                                 const float4 *__restrict__ egrad, float L, const float *__restrict__ dZ,
                                 float *__restrict__ dhv)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)V * HC;
         t += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / HC), c = (int)(t % HC);
        float s = 0.0f;
        for (int q = voff[v]; q < voff[v + 1]; q++) {
            const int ek = vinc[q], e = ek >> 2, k = ek & 3;
            const float4 g = egrad[e];
            const float gx = k == 0 ? g.x : (k == 1 ? g.z : -(g.x + g.z));
            const float gy = k == 0 ? g.y : (k == 1 ? g.w : -(g.y + g.w));
            const float *dz = dZ + (size_t)e * 3 * HC;
            s += gx * dz[HC + c] + gy * dz[2 * HC + c];
        }
        dhv[t] += L * s;
    }
}

// Z_v = [h_v, sum_{(e,k) at v} A_e h_e / sum A_e], rebuilt for the backward pass
__global__ void k_msg_vert(int V, const int *__restrict__ voff, const int *__restrict__ vinc,
                           const float *__restrict__ earea, const float *__restrict__ vinvA,
                           const float *__restrict__ hv, const float *__restrict__ he, float *__restrict__ Z)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)V * HC;
         t += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(t / HC), c = (int)(t % HC);
        float s = 0.0f;
        for (int q = voff[v]; q < voff[v + 1]; q++) {
            const int e = vinc[q] >> 2;
            s = msg_vert_acc(s, earea[e], he[(size_t)e * HC + c]);
        }
        float *z = Z + (size_t)v * 2 * HC;
        z[c] = bf16_value(hv[t]);
        z[HC + c] = bf16_value(msg_vert_mean(s, vinvA[v]));
    }
}

// dh_v += dZ_v[:, 0:64]
__global__ void k_msg_vert_adj_v(int V, const float *__restrict__ dZ, float *__restrict__ dhv)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)V * HC;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t v = t / HC;
        dhv[t] += dZ[v * 2 * HC + t % HC];
    }
}

// dh_e += sum_k A_e / (sum A)_{v_k} dZ_v[v_k][64 + c]
__global__ void k_msg_vert_adj_e(int E, const int4 *__restrict__ etri, const float *__restrict__ earea,
                                 const float *__restrict__ vinvA, const float *__restrict__ dZ, float *__restrict__ dhe)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)E * HC;
         t += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(t / HC), c = (int)(t % HC);
        const int4 v = etri[e];
        const float a = earea[e];
        dhe[t] += a * (vinvA[v.x] * dZ[(size_t)v.x * 2 * HC + HC + c] + vinvA[v.y] * dZ[(size_t)v.y * 2 * HC + HC + c] +
                       vinvA[v.z] * dZ[(size_t)v.z * 2 * HC + HC + c]);
    }
}

// ------------------------------------------------------------------------- data

// Element arrays (element order of the library) from the owned slots.
__global__ void k_build_elems(const int4 *__restrict__ sv, const float4 *__restrict__ sg, const float4 *__restrict__ sc,
                              int nslot, int4 *__restrict__ etri, float4 *__restrict__ egrad, float *__restrict__ earea,
                              float *__restrict__ eH0, float *__restrict__ ef, int *__restrict__ eslot)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const int4 v = sv[s];
        if (v.w < 0) continue;
        etri[v.w] = make_int4(v.x, v.y, v.z, 0);
        egrad[v.w] = sg[s];
        const float4 c = sc[s];
        earea[v.w] = c.x;
        eH0[v.w] = c.y;
        ef[v.w] = c.z;
        eslot[v.w] = s;
    }
}

__device__ __forceinline__ float safe_inv(float s) { return s > 0.0f ? 1.0f / s : 0.0f; }

// Features of one sample: x_v [V][2], x_e [E][6].
__global__ void k_features(int V, int E, const float *__restrict__ eta, const float *__restrict__ U,
                           const float *__restrict__ R, const float *__restrict__ h0v, const float *__restrict__ eH0,
                           const float *__restrict__ ef, const float *__restrict__ sc, float *__restrict__ xv,
                           float *__restrict__ xe)
{
    const int n = max(V, E);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < V) {
            xv[2 * i] = eta[i] * safe_inv(sc[S_ETA]);
            xv[2 * i + 1] = h0v[i] * safe_inv(sc[S_H]);
        }
        if (i < E) {
            float *x = xe + 6 * (size_t)i;
            x[0] = U[2 * i] * safe_inv(sc[S_U]);
            x[1] = U[2 * i + 1] * safe_inv(sc[S_U]);
            x[2] = R[2 * i] * safe_inv(sc[S_R]);
            x[3] = R[2 * i + 1] * safe_inv(sc[S_R]);
            x[4] = ef[i] * safe_inv(sc[S_F]);
            x[5] = eH0[i] * safe_inv(sc[S_H]);
        }
    }
}

// Loss (mean squared error of the normalized outputs) and its gradient.
// te: [E][4] raw increments (<<U>>-U, U^M-U); tv: [V] raw eta_bar - eta.
__global__ void __launch_bounds__(256)
k_loss(int V, int E, const float *__restrict__ oe, const float *__restrict__ ov, const float *__restrict__ te,
       const float *__restrict__ tv, const float *__restrict__ sc, float *__restrict__ doe, float *__restrict__ dov,
       double *__restrict__ part)
{
    __shared__ double sh[8];
    const float iU = safe_inv(sc[S_OU]), iE = safe_inv(sc[S_OETA]);
    double acc = 0.0;
    const double we = 1.0 / (4.0 * E), wv = 1.0 / (double)V;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * E; i += gridDim.x * blockDim.x) {
        const float d = oe[i] - te[i] * iU;
        acc += we * (double)d * d;
        if (doe) doe[i] = (float)(2.0 * we) * d;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
        const float d = ov[i] - tv[i] * iE;
        acc += wv * (double)d * d;
        if (dov) dov[i] = (float)(2.0 * wv) * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_sum_parts(const double *__restrict__ part, int n, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += part[i];
        out[0] = s;
    }
}

// Adam with bias correction; matrices are stored again as bfloat16 for the next forward.
__global__ void k_adam(int n, float *__restrict__ w, __nv_bfloat16 *__restrict__ w16, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[i] = wi;
        w16[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void k_to_bf16(int n, const float *__restrict__ w, __nv_bfloat16 *__restrict__ w16)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w16[i] = __float2bfloat16_rn(w[i]);
}

// Copy the context's current state (library order) into sample arrays.
__global__ void k_take_state(int V, int E, const float *__restrict__ eta, const float2 *__restrict__ Us,
                             const float2 *__restrict__ Rs, const int *__restrict__ eslot, float *__restrict__ d_eta,
                             float *__restrict__ d_U, float *__restrict__ d_R)
{
    const int n = max(V, E);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < V) d_eta[i] = eta[i];
        if (i < E) {
            const int s = eslot[i];
            const float2 u = Us[s], r = Rs[s];
            d_U[2 * i] = u.x;
            d_U[2 * i + 1] = u.y;
            d_R[2 * i] = r.x;
            d_R[2 * i + 1] = r.y;
        }
    }
}

// Targets after a plain step: <<U>> - U^0, U^M - U^0 per element; eta_bar - eta^0 per vertex.
__global__ void k_take_targets(int V, int E, const float *__restrict__ eta_sum, float inv_M,
                               const float2 *__restrict__ Us, const float2 *__restrict__ Umean,
                               const int *__restrict__ eslot, const float *__restrict__ in_eta,
                               const float *__restrict__ in_U, float *__restrict__ te, float *__restrict__ tv)
{
    const int n = max(V, E);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < V) tv[i] = eta_sum[i] * inv_M - in_eta[i];
        if (i < E) {
            const float2 um = Umean[i], u = Us[eslot[i]];
            te[4 * i] = um.x - in_U[2 * i];
            te[4 * i + 1] = um.y - in_U[2 * i + 1];
            te[4 * i + 2] = u.x - in_U[2 * i];
            te[4 * i + 3] = u.y - in_U[2 * i + 1];
        }
    }
}

// A sample given in caller order (doubles) into library order (floats).
__global__ void k_sample_from_caller(int V, int E, const int *__restrict__ vperm, const int *__restrict__ eperm,
                                     const double *__restrict__ eta, const double *__restrict__ U,
                                     const double *__restrict__ R, const double *__restrict__ tum,
                                     const double *__restrict__ tuM, const double *__restrict__ teb,
                                     float *__restrict__ d_eta, float *__restrict__ d_U, float *__restrict__ d_R,
                                     float *__restrict__ te, float *__restrict__ tv)
{
    const int n = max(V, E);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < V) {
            const int c = vperm[i];
            d_eta[i] = (float)eta[c];
            tv[i] = (float)teb[c];
        }
        if (i < E) {
            const int c = eperm[i];
            d_U[2 * i] = (float)U[2 * c];
            d_U[2 * i + 1] = (float)U[2 * c + 1];
            d_R[2 * i] = (float)R[2 * c];
            d_R[2 * i + 1] = (float)R[2 * c + 1];
            te[4 * i] = (float)tum[2 * c];
            te[4 * i + 1] = (float)tum[2 * c + 1];
            te[4 * i + 2] = (float)tuM[2 * c];
            te[4 * i + 3] = (float)tuM[2 * c + 1];
        }
    }
}

// Sums of squares of the sample quantities (for the scales): out[8] per block.
__global__ void __launch_bounds__(256)
k_sumsq(int V, int E, const float *__restrict__ eta, const float *__restrict__ U, const float *__restrict__ R,
        const float *__restrict__ te, const float *__restrict__ tv, double *__restrict__ part)
{
    __shared__ double sh[6][8];
    double a[6] = {0, 0, 0, 0, 0, 0};   // eta, U, R, out_U (both increments), out_eta, count guard
    const int n = max(V, E);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < V) {
            a[0] += (double)eta[i] * eta[i];
            a[4] += (double)tv[i] * tv[i];
        }
        if (i < E) {
            a[1] += (double)U[2 * i] * U[2 * i] + (double)U[2 * i + 1] * U[2 * i + 1];
            a[2] += (double)R[2 * i] * R[2 * i] + (double)R[2 * i + 1] * R[2 * i + 1];
            for (int q = 0; q < 4; q++) a[3] += (double)te[4 * i + q] * te[4 * i + q];
        }
    }
    for (int q = 0; q < 5; q++) {
        double x = a[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[threadIdx.x][w];
        part[blockIdx.x * 8 + threadIdx.x] = s;
    }
}

// --- inference: apply a prediction and check the summed momentum equation

// <<U>>, U^M (all slot copies) and eta_bar from the network outputs.
__global__ void k_apply_elems(int E, int nslot, const int4 *__restrict__ sv, const float *__restrict__ oe,
                              const float *__restrict__ sc, const float *__restrict__ U0e, float2 *__restrict__ Us,
                              float2 *__restrict__ Umean)
{
    const float sU = sc[S_OU];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslot; s += gridDim.x * blockDim.x) {
        const int w = sv[s].w, e = w >= 0 ? w : -1 - w;
        const float *o = oe + 4 * (size_t)e;
        const float ux = U0e[2 * e], uy = U0e[2 * e + 1];
        Us[s] = make_float2(ux + sU * o[2], uy + sU * o[3]);
        if (w >= 0) Umean[w] = make_float2(ux + sU * o[0], uy + sU * o[1]);
    }
}

// eta^{n+1} = eta^n - tau div <<U>> (median-dual divergence, as the plain vertex pass)
// and eta_bar = eta^n + s_oeta o_v.
__global__ void k_apply_verts(int V, const int *__restrict__ voff, const int *__restrict__ vinc,
                              const float4 *__restrict__ egrad, const float *__restrict__ earea,
                              const float *__restrict__ inv_av, const float2 *__restrict__ Umean,
                              const float *__restrict__ ov, const float *__restrict__ sc, float tau,
                              const float *__restrict__ eta0, float *__restrict__ eta1, float *__restrict__ etabar)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int q = voff[v]; q < voff[v + 1]; q++) {
            const int ek = vinc[q], e = ek >> 2, k = ek & 3;
            const float4 g = egrad[e];
            const float gx = k == 0 ? g.x : (k == 1 ? g.z : -(g.x + g.z));
            const float gy = k == 0 ? g.y : (k == 1 ? g.w : -(g.y + g.w));
            const float2 u = Umean[e];
            s += tau * earea[e] * (u.x * gx + u.y * gy);
        }
        eta1[v] = eta0[v] + s * inv_av[v];
        etabar[v] = eta0[v] + sc[S_OETA] * ov[v];
    }
}

// Residual of the summed momentum equation per element,
//   r = U^M - U^0 + tau [ f e_z x S' + g H grad(eta_bar) - R ],
//   S' = <<U>> - (theta/M)(U^M - U^0) + (U^0 - U^M)/(2M);
// part[b] = (sum A |r|^2, sum A |U^M - U^0|^2) per block.
__global__ void __launch_bounds__(256)
k_residual(int E, const int4 *__restrict__ etri, const float4 *__restrict__ egrad, const float *__restrict__ earea,
           const float *__restrict__ eH0, const float *__restrict__ ef, const int *__restrict__ eslot,
           const float2 *__restrict__ Us, const float2 *__restrict__ Umean, const float *__restrict__ U0e,
           const float *__restrict__ R0e, const float *__restrict__ etabar, float tau, float g, float theta,
           float M, int nonlinear_h, double *__restrict__ part)
{
    __shared__ double sh[2][8];
    double a = 0.0, b = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const int4 v = etri[e];
        const float4 gr = egrad[e];
        const float e0 = etabar[v.x], e1 = etabar[v.y], e2 = etabar[v.z];
        const float d0 = e0 - e2, d1 = e1 - e2;
        const float gx = d0 * gr.x + d1 * gr.z, gy = d0 * gr.y + d1 * gr.w;
        float H = eH0[e];
        if (nonlinear_h) H += (e0 + e1 + e2) * (1.0f / 3.0f);
        const float2 uM = Us[eslot[e]], um = Umean[e];
        const float dux = uM.x - U0e[2 * e], duy = uM.y - U0e[2 * e + 1];
        const float spx = um.x - theta / M * dux - dux / (2.0f * M);
        const float spy = um.y - theta / M * duy - duy / (2.0f * M);
        const float f = ef[e];
        const float rx = dux + tau * (-f * spy + g * H * gx - R0e[2 * e]);
        const float ry = duy + tau * (f * spx + g * H * gy - R0e[2 * e + 1]);
        const double A = earea[e];
        a += A * ((double)rx * rx + (double)ry * ry);
        b += A * ((double)dux * dux + (double)duy * duy);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a;
        sh[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            sa += sh[0][w];
            sb += sh[1][w];
        }
        part[2 * blockIdx.x] = sa;
        part[2 * blockIdx.x + 1] = sb;
    }
}

int grid1(size_t n, int threads = 256)
{
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)std::max<size_t>(b, 1);
}

}  // namespace

struct Layer {
    int K, C;        // matrix is K x C
    size_t w, b;     // offsets in the parameter vector
    long tc = -1;    // offset of the tensor-core copy of W (packed W^T) in Surrogate::wtc, or -1
};

struct Surrogate {
    int V = 0, E = 0;
    // graph
    int4 *etri = nullptr;
    float4 *egrad = nullptr;
    float *earea = nullptr, *eH0 = nullptr, *ef = nullptr, *vinvA = nullptr;
    int *eslot = nullptr, *voff = nullptr, *vinc = nullptr;
    // parameters
    std::vector<Layer> L;    // Wv0, We0, We1, Wv1, We2, Wv2, We3, Wv3, Weo, Wvo
    int nparam = 0;
    float *w32 = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    __nv_bfloat16 *w16 = nullptr;
    __nv_bfloat16 *wtc = nullptr;   // packed copies of the tensor-core layers' weights
    size_t ntc = 0;
    long adam_t = 0;
    double lr = 1e-3, b1 = 0.9, b2 = 0.999, eps = 1e-8;
    float *scales = nullptr;   // device [8]
    double scales_h[NSCALE] = {1, 1, 1, 1, 1, 1, 1, 1};
    // activations
    float *xv = nullptr, *xe = nullptr;
    float *hv[NL + 1] = {}, *he[NL + 1] = {}, *yv[NL] = {}, *ye[NL] = {};
    float *oe = nullptr, *ov = nullptr, *ze = nullptr, *zv = nullptr;
    float *dze = nullptr, *dzv = nullptr, *dhe = nullptr, *dhv = nullptr, *dae = nullptr, *dav = nullptr;
    float *doe = nullptr, *dov = nullptr;
    float *partial = nullptr;
    size_t partial_len = 0;
    double *red = nullptr;      // reductions
    // dataset
    long cap = 0;
    float *d_eta = nullptr, *d_U = nullptr, *d_R = nullptr, *d_te = nullptr, *d_tv = nullptr;
    // inference
    float *cur_eta = nullptr, *cur_U = nullptr, *cur_R = nullptr, *etabar = nullptr;
    float *save_eta = nullptr;
    float2 *save_U = nullptr;
    double *stage = nullptr;    // host samples in transit: 2 V + 8 E doubles
    size_t smem_mm = 0;
    unsigned *status = nullptr; // the context's device status word (timeout bit of the tensor-core waits)
};

void surrogate_release(sesw_ctx *c)
{
    // device memory belongs to the context's allocation list and is freed with it
    delete c->sur;
    c->sur = nullptr;
}

namespace {

#define SCK(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return sesw::ctx_fail_cuda(c, #call, e_);   \
    } while (0)

template <class T>
int salloc(sesw_ctx *c, T **p, size_t n)
{
    *p = (T *)ctx_alloc(c, sizeof(T) * std::max<size_t>(n, 1));
    if (!*p) return ctx_fail(c, SESW_ENOMEM, "device allocation failed for the surrogate");
    return SESW_OK;
}

#define STRY(x)                        \
    do {                               \
        int r_ = (x);                  \
        if (r_ != SESW_OK) return r_;  \
    } while (0)

cudaError_t mm(Surrogate &S, cudaStream_t st, int N, int Kin, int P, const float *X, const __nv_bfloat16 *W,
               int trans, const float *bias, int act, const float *res, float *Y)
{

    const size_t smem = sizeof(float) * ((size_t)TILE_ROWS * (Kin + 1) + (size_t)Kin * P);
    const int grid = (N + TILE_ROWS - 1) / TILE_ROWS;
    if (grid == 0) return cudaSuccess;
    if (P <= 64)
        k_mm<4><<<grid, 256, smem, st>>>(N, Kin, P, X, W, trans, bias, act, res, Y);
    else
        k_mm<12><<<grid, 256, smem, st>>>(N, Kin, P, X, W, trans, bias, act, res, Y);
    return cudaGetLastError();
}

// Forward of message layer ly (kind 0: element rows from h_e[l] and h_v[l]; kind 1: vertex rows
// from h_v[l] and h_e[l + 1]) on the tensor cores, the message gather fused into the layer:
// writes Y and h_next = h + Y.
cudaError_t msg_layer(Surrogate &S, cudaStream_t st, const Layer &ly, int kind, const float *hself,
                      const float *hother, float *Y, float *hnext)
{
    if (ly.tc < 0) return cudaErrorInvalidValue;
    MsgLayerArgs a;
    a.kind = kind;
    a.N = kind == 0 ? S.E : S.V;
    a.etri = S.etri;
    a.egrad = S.egrad;
    a.L = (float)S.scales_h[S_L];
    a.voff = S.voff;
    a.vinc = S.vinc;
    a.earea = S.earea;
    a.vinvA = S.vinvA;
    a.hself = hself;
    a.hother = hother;
    a.Y = Y;
    a.hnext = hnext;
    return launch_msg_layer_tc(a, S.wtc + ly.tc, S.w32 + ly.b, S.status, st);
}

// Refresh the packed tensor-core copies after the bfloat16 weights changed.
cudaError_t pack_tc(Surrogate &S, cudaStream_t st)
{
    for (const Layer &ly : S.L)
        if (ly.tc >= 0) {
            const cudaError_t e = pack_linear_tc(ly.K, S.w16 + ly.w, S.wtc + ly.tc, st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// gradient of layer l's matrix and bias from its input Z [N][K] and dA [N][C]; the message
// layers (inputs rounded to bfloat16 values, 64 outputs) on the tensor cores
cudaError_t wgrad(Surrogate &S, cudaStream_t st, const Layer &ly, int N, const float *Z, const float *dA)
{
    // the small layers have few outputs per block, so their blocks take fewer rows (more blocks
    // in flight); the partial buffer holds ceil(N / 2048) partials of the largest layer
    const int len = ly.K * ly.C + ly.C;
    int rows = 2048;
    if (ly.tc < 0)
        while (rows > 128 && (size_t)((N + rows / 2 - 1) / (rows / 2)) * len <= S.partial_len) rows /= 2;
    const int nb = std::max(1, (N + rows - 1) / rows);
    if (ly.tc >= 0) {
        const cudaError_t e = launch_wgrad_tc(N, ly.K, rows, Z, dA, S.partial, S.status, st);
        if (e != cudaSuccess) return e;
    } else {
        // the staged tiles hold WG_ROWS rows of at most HC values; a thread owns at most 2 outputs
        if (ly.K > HC || ly.C > HC || ly.K * ly.C + ly.C > 512) return cudaErrorInvalidValue;
        k_wgrad_small<<<nb, 256, 0, st>>>(N, ly.K, ly.C, Z, dA, rows, S.partial);
    }
    k_reduce_partials<<<grid1(len), 256, 0, st>>>(S.partial, nb, len, S.grad + ly.w, S.grad + ly.b, ly.K * ly.C);
    return cudaGetLastError();
}

// dZ = dA W^T of a message layer (the gradient with respect to its inputs), on the tensor cores
cudaError_t dgrad(Surrogate &S, cudaStream_t st, const Layer &ly, int N, const float *dA, float *dZ)
{
    if (ly.tc >= 0) return launch_dgrad_tc(N, ly.K, dA, S.w16 + ly.w, dZ, S.status, st);
    return mm(S, st, N, ly.C, ly.K, dA, S.w16 + ly.w, 1, nullptr, 0, nullptr, dZ);
}

// forward of one sample whose features are in S.xv, S.xe; keep_y keeps each message layer's
// activation Y for the backward pass (inference does without it)
cudaError_t forward(Surrogate &S, cudaStream_t st, bool keep_y = true)
{
    cudaError_t e;
    const Layer &lv0 = S.L[0], &le0 = S.L[1];
    if ((e = mm(S, st, S.V, 2, HC, S.xv, S.w16 + lv0.w, 0, S.w32 + lv0.b, 1, nullptr, S.hv[0])) != cudaSuccess) return e;
    if ((e = mm(S, st, S.E, 6, HC, S.xe, S.w16 + le0.w, 0, S.w32 + le0.b, 1, nullptr, S.he[0])) != cudaSuccess) return e;
    for (int l = 0; l < NL; l++) {
        const Layer &le = S.L[2 + 2 * l], &lv = S.L[3 + 2 * l];
        // h_e(l+1) = h_e(l) + y_e(l), then h_v(l+1) = h_v(l) + y_v(l) from h_e(l+1)
        if ((e = msg_layer(S, st, le, 0, S.he[l], S.hv[l], keep_y ? S.ye[l] : nullptr, S.he[l + 1])) != cudaSuccess)
            return e;
        if ((e = msg_layer(S, st, lv, 1, S.hv[l], S.he[l + 1], keep_y ? S.yv[l] : nullptr, S.hv[l + 1])) !=
            cudaSuccess)
            return e;
    }
    const Layer &leo = S.L[2 + 2 * NL], &lvo = S.L[3 + 2 * NL];
    if ((e = mm(S, st, S.E, HC, 4, S.he[NL], S.w16 + leo.w, 0, S.w32 + leo.b, 0, nullptr, S.oe)) != cudaSuccess) return e;
    if ((e = mm(S, st, S.V, HC, 1, S.hv[NL], S.w16 + lvo.w, 0, S.w32 + lvo.b, 0, nullptr, S.ov)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// backward from S.doe, S.dov to S.grad (overwritten)
cudaError_t backward(Surrogate &S, cudaStream_t st)
{
    const float Ls = (float)S.scales_h[S_L];
    cudaError_t e;
    const Layer &leo = S.L[2 + 2 * NL], &lvo = S.L[3 + 2 * NL];
    if ((e = wgrad(S, st, leo, S.E, S.he[NL], S.doe)) != cudaSuccess) return e;
    if ((e = wgrad(S, st, lvo, S.V, S.hv[NL], S.dov)) != cudaSuccess) return e;
    if ((e = mm(S, st, S.E, 4, HC, S.doe, S.w16 + leo.w, 1, nullptr, 0, nullptr, S.dhe)) != cudaSuccess) return e;
    if ((e = mm(S, st, S.V, 1, HC, S.dov, S.w16 + lvo.w, 1, nullptr, 0, nullptr, S.dhv)) != cudaSuccess) return e;
    for (int l = NL - 1; l >= 0; l--) {
        const Layer &le = S.L[2 + 2 * l], &lv = S.L[3 + 2 * l];
        // vertex update of layer l
        k_tanh_bwd<<<grid1((size_t)S.V * HC), 256, 0, st>>>((size_t)S.V * HC, S.dhv, S.yv[l], S.dav);
        k_msg_vert<<<grid1((size_t)S.V * HC), 256, 0, st>>>(S.V, S.voff, S.vinc, S.earea, S.vinvA, S.hv[l], S.he[l + 1],
                                                            S.zv);
        if ((e = wgrad(S, st, lv, S.V, S.zv, S.dav)) != cudaSuccess) return e;
        if ((e = dgrad(S, st, lv, S.V, S.dav, S.dzv)) != cudaSuccess) return e;
        k_msg_vert_adj_v<<<grid1((size_t)S.V * HC), 256, 0, st>>>(S.V, S.dzv, S.dhv);
        k_msg_vert_adj_e<<<grid1((size_t)S.E * HC), 256, 0, st>>>(S.E, S.etri, S.earea, S.vinvA, S.dzv, S.dhe);
        // element update of layer l
        k_tanh_bwd<<<grid1((size_t)S.E * HC), 256, 0, st>>>((size_t)S.E * HC, S.dhe, S.ye[l], S.dae);
        k_msg_elem<<<grid1((size_t)S.E * HC), 256, 0, st>>>(S.E, S.etri, S.egrad, Ls, S.he[l], S.hv[l], S.ze);
        if ((e = wgrad(S, st, le, S.E, S.ze, S.dae)) != cudaSuccess) return e;
        if ((e = dgrad(S, st, le, S.E, S.dae, S.dze)) != cudaSuccess) return e;
        k_msg_elem_adj_e<<<grid1((size_t)S.E * HC), 256, 0, st>>>(S.E, S.dze, S.dhe);
        k_msg_elem_adj_v<<<grid1((size_t)S.V * HC), 256, 0, st>>>(S.V, S.voff, S.vinc, S.egrad, Ls, S.dze, S.dhv);
    }
    const Layer &lv0 = S.L[0], &le0 = S.L[1];
    k_tanh_bwd<<<grid1((size_t)S.V * HC), 256, 0, st>>>((size_t)S.V * HC, S.dhv, S.hv[0], S.dav);
    if ((e = wgrad(S, st, lv0, S.V, S.xv, S.dav)) != cudaSuccess) return e;
    k_tanh_bwd<<<grid1((size_t)S.E * HC), 256, 0, st>>>((size_t)S.E * HC, S.dhe, S.he[0], S.dae);
    if ((e = wgrad(S, st, le0, S.E, S.xe, S.dae)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// features of sample i of the dataset into xv, xe
void features_of(Surrogate &S, sesw_ctx *c, long i)
{
    k_features<<<grid1(std::max(S.V, S.E)), 256, 0, c->stream>>>(
        S.V, S.E, S.d_eta + (size_t)i * S.V, S.d_U + (size_t)i * 2 * S.E, S.d_R + (size_t)i * 2 * S.E, c->dm.h0_v,
        S.eH0, S.ef, S.scales, S.xv, S.xe);
}

cudaError_t loss_of(Surrogate &S, sesw_ctx *c, long i, bool want_grad, double *dst)
{
    const int nb = 152 * 4;
    k_loss<<<nb, 256, 0, c->stream>>>(S.V, S.E, S.oe, S.ov, S.d_te + (size_t)i * 4 * S.E, S.d_tv + (size_t)i * S.V,
                                      S.scales, want_grad ? S.doe : nullptr, want_grad ? S.dov : nullptr, S.red + 16);
    k_sum_parts<<<1, 32, 0, c->stream>>>(S.red + 16, nb, dst);
    return cudaGetLastError();
}

}  // namespace

}  // namespace sesw

using sesw::Surrogate;

extern "C" {

int sesw_surrogate_init(sesw_ctx *c, int32_t capacity, int32_t seed)
{
    if (!c) return SESW_EINVAL;
    if (!c->have_mesh) return sesw::ctx_fail(c, SESW_ESTATE, "upload a mesh before creating the surrogate");
    if (c->nbasin != 1) return sesw::ctx_fail(c, SESW_EINVAL, "the surrogate works on a single mesh, not a batch");
    if (capacity < 1) return sesw::ctx_fail(c, SESW_EINVAL, "capacity must be >= 1");
    cudaSetDevice(c->device);
    sesw::surrogate_release(c);
    Surrogate *Sp = new (std::nothrow) Surrogate();
    if (!Sp) return sesw::ctx_fail(c, SESW_ENOMEM, "host allocation failed");
    c->sur = Sp;
    Surrogate &S = *Sp;
    const int V = c->dm.nv, E = c->dm.ne;
    S.V = V;
    S.status = c->ds.status;
    S.E = E;
    S.cap = capacity;
    // graph
    STRY(sesw::salloc(c, &S.etri, E));
    STRY(sesw::salloc(c, &S.egrad, E));
    STRY(sesw::salloc(c, &S.earea, E));
    STRY(sesw::salloc(c, &S.eH0, E));
    STRY(sesw::salloc(c, &S.ef, E));
    STRY(sesw::salloc(c, &S.eslot, E));
    sesw::k_build_elems<<<sesw::grid1(c->dm.nslot), 256, 0, c->stream>>>(c->dm.slot_v, c->dm.slot_g, c->dm.slot_c,
                                                                          c->dm.nslot, S.etri, S.egrad, S.earea, S.eH0,
                                                                          S.ef, S.eslot);
    SCK(cudaGetLastError());
    std::vector<int4> etri(E);
    std::vector<float> earea(E);
    SCK(cudaMemcpyAsync(etri.data(), S.etri, sizeof(int4) * E, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaMemcpyAsync(earea.data(), S.earea, sizeof(float) * E, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    std::vector<int> off(V + 1, 0), inc(3 * (size_t)E);
    std::vector<double> asum(V, 0.0);
    for (int e = 0; e < E; e++) {
        const int cv[3] = {etri[e].x, etri[e].y, etri[e].z};
        for (int k = 0; k < 3; k++) {
            off[cv[k] + 1]++;
            asum[cv[k]] += earea[e];
        }
    }
    for (int v = 0; v < V; v++) off[v + 1] += off[v];
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int e = 0; e < E; e++) {
            const int cv[3] = {etri[e].x, etri[e].y, etri[e].z};
            for (int k = 0; k < 3; k++) inc[fill[cv[k]]++] = (e << 2) | k;
        }
    }
    std::vector<float> vinvA(V);
    for (int v = 0; v < V; v++) vinvA[v] = asum[v] > 0.0 ? (float)(1.0 / asum[v]) : 0.0f;
    STRY(sesw::salloc(c, &S.voff, V + 1));
    STRY(sesw::salloc(c, &S.vinc, 3 * (size_t)E));
    STRY(sesw::salloc(c, &S.vinvA, V));
    SCK(cudaMemcpyAsync(S.voff, off.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, c->stream));
    SCK(cudaMemcpyAsync(S.vinc, inc.data(), sizeof(int) * inc.size(), cudaMemcpyHostToDevice, c->stream));
    SCK(cudaMemcpyAsync(S.vinvA, vinvA.data(), sizeof(float) * V, cudaMemcpyHostToDevice, c->stream));
    // parameters: Wv0 (2x64), We0 (6x64), then per layer We (192x64), Wv (128x64), then Weo (64x4), Wvo (64x1)
    auto add = [&](int K, int C) {
        sesw::Layer ly;
        ly.K = K;
        ly.C = C;
        ly.w = S.nparam;
        S.nparam += K * C;
        ly.b = S.nparam;
        S.nparam += C;
        if (sesw::linear_tc_supported(K, C)) {
            ly.tc = (long)S.ntc;
            S.ntc += sesw::linear_tc_packed_elems(K);
        }
        S.L.push_back(ly);
    };
    add(2, sesw::HC);
    add(6, sesw::HC);
    for (int l = 0; l < sesw::NL; l++) {
        add(3 * sesw::HC, sesw::HC);
        add(2 * sesw::HC, sesw::HC);
    }
    add(sesw::HC, 4);
    add(sesw::HC, 1);
    STRY(sesw::salloc(c, &S.w32, S.nparam));
    STRY(sesw::salloc(c, &S.grad, S.nparam));
    STRY(sesw::salloc(c, &S.am, S.nparam));
    STRY(sesw::salloc(c, &S.av, S.nparam));
    STRY(sesw::salloc(c, &S.w16, S.nparam));
    STRY(sesw::salloc(c, &S.wtc, S.ntc));
    {
        // Glorot-uniform matrices, zero biases, from a seeded generator
        std::vector<float> w(S.nparam, 0.0f);
        std::mt19937_64 rng((uint64_t)seed * 0x9E3779B97F4A7C15ull + 12345u);
        for (const auto &ly : S.L) {
            const double a = sqrt(6.0 / (ly.K + ly.C));
            std::uniform_real_distribution<double> U(-a, a);
            for (int i = 0; i < ly.K * ly.C; i++) w[ly.w + i] = (float)U(rng);
        }
        SCK(cudaMemcpyAsync(S.w32, w.data(), sizeof(float) * S.nparam, cudaMemcpyHostToDevice, c->stream));
        SCK(cudaMemsetAsync(S.am, 0, sizeof(float) * S.nparam, c->stream));
        SCK(cudaMemsetAsync(S.av, 0, sizeof(float) * S.nparam, c->stream));
        sesw::k_to_bf16<<<sesw::grid1(S.nparam), 256, 0, c->stream>>>(S.nparam, S.w32, S.w16);
        SCK(sesw::pack_tc(S, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
    }
    STRY(sesw::salloc(c, &S.scales, sesw::NSCALE));
    {
        const float ones[sesw::NSCALE] = {1, 1, 1, 1, 1, 1, 1, 1};
        SCK(cudaMemcpyAsync(S.scales, ones, sizeof ones, cudaMemcpyHostToDevice, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
    }
    // activations
    const size_t vh = (size_t)V * sesw::HC, eh = (size_t)E * sesw::HC;
    STRY(sesw::salloc(c, &S.xv, 2 * (size_t)V));
    STRY(sesw::salloc(c, &S.xe, 6 * (size_t)E));
    for (int l = 0; l <= sesw::NL; l++) {
        STRY(sesw::salloc(c, &S.hv[l], vh));
        STRY(sesw::salloc(c, &S.he[l], eh));
    }
    for (int l = 0; l < sesw::NL; l++) {
        STRY(sesw::salloc(c, &S.yv[l], vh));
        STRY(sesw::salloc(c, &S.ye[l], eh));
    }
    STRY(sesw::salloc(c, &S.oe, 4 * (size_t)E));
    STRY(sesw::salloc(c, &S.ov, (size_t)V));
    STRY(sesw::salloc(c, &S.ze, 3 * eh));
    STRY(sesw::salloc(c, &S.zv, 2 * vh));
    STRY(sesw::salloc(c, &S.dze, 3 * eh));
    STRY(sesw::salloc(c, &S.dzv, 2 * vh));
    STRY(sesw::salloc(c, &S.dhe, eh));
    STRY(sesw::salloc(c, &S.dhv, vh));
    STRY(sesw::salloc(c, &S.dae, eh));
    STRY(sesw::salloc(c, &S.dav, vh));
    STRY(sesw::salloc(c, &S.doe, 4 * (size_t)E));
    STRY(sesw::salloc(c, &S.dov, (size_t)V));
    const int nbmax = std::max(1, (std::max(V, E) + 2047) / 2048);
    S.partial_len = (size_t)nbmax * (3 * sesw::HC * sesw::HC + sesw::HC);
    STRY(sesw::salloc(c, &S.partial, S.partial_len));
    STRY(sesw::salloc(c, &S.red, 16 + 152 * 4 * 8));
    // dataset and inference buffers
    STRY(sesw::salloc(c, &S.d_eta, (size_t)capacity * V));
    STRY(sesw::salloc(c, &S.d_U, (size_t)capacity * 2 * E));
    STRY(sesw::salloc(c, &S.d_R, (size_t)capacity * 2 * E));
    STRY(sesw::salloc(c, &S.d_te, (size_t)capacity * 4 * E));
    STRY(sesw::salloc(c, &S.d_tv, (size_t)capacity * V));
    STRY(sesw::salloc(c, &S.cur_eta, (size_t)V));
    STRY(sesw::salloc(c, &S.cur_U, 2 * (size_t)E));
    STRY(sesw::salloc(c, &S.cur_R, 2 * (size_t)E));
    STRY(sesw::salloc(c, &S.etabar, (size_t)V));
    STRY(sesw::salloc(c, &S.save_eta, (size_t)V));
    STRY(sesw::salloc(c, &S.save_U, (size_t)c->dm.nslot));
    STRY(sesw::salloc(c, &S.stage, 2 * (size_t)V + 8 * (size_t)E));
    // matrix kernels need up to (64 x 193 + 192 x 64) floats of shared memory
    S.smem_mm = sizeof(float) * (64 * (3 * sesw::HC + 1) + 3 * sesw::HC * sesw::HC);
    SCK(cudaFuncSetAttribute(sesw::k_mm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem_mm));
    SCK(cudaFuncSetAttribute(sesw::k_mm<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem_mm));
    SCK(cudaStreamSynchronize(c->stream));
    return SESW_OK;
}

static int need_sur(sesw_ctx *c)
{
    if (!c) return SESW_EINVAL;
    if (!c->sur) return sesw::ctx_fail(c, SESW_ESTATE, "create the surrogate first (sesw_surrogate_init)");
    cudaSetDevice(c->device);
    return SESW_OK;
}

int sesw_surrogate_nparam(sesw_ctx *c, int64_t *n)
{
    STRY(need_sur(c));
    if (n) *n = c->sur->nparam;
    return SESW_OK;
}

int sesw_surrogate_weights(sesw_ctx *c, float *get, const float *set)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (set) {
        SCK(cudaMemcpyAsync(S.w32, set, sizeof(float) * S.nparam, cudaMemcpyHostToDevice, c->stream));
        sesw::k_to_bf16<<<sesw::grid1(S.nparam), 256, 0, c->stream>>>(S.nparam, S.w32, S.w16);
        SCK(cudaGetLastError());
        SCK(sesw::pack_tc(S, c->stream));
    }
    if (get) SCK(cudaMemcpyAsync(get, S.w32, sizeof(float) * S.nparam, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    return SESW_OK;
}

int sesw_surrogate_scales(sesw_ctx *c, double *get, const double *set)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (set) {
        float f[sesw::NSCALE];
        for (int i = 0; i < sesw::NSCALE; i++) {
            if (!(set[i] > 0.0) || !std::isfinite(set[i])) return sesw::ctx_fail(c, SESW_EINVAL, "scales must be positive");
            S.scales_h[i] = set[i];
            f[i] = (float)set[i];
        }
        SCK(cudaMemcpyAsync(S.scales, f, sizeof f, cudaMemcpyHostToDevice, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
    }
    if (get) memcpy(get, S.scales_h, sizeof S.scales_h);
    return SESW_OK;
}

int sesw_surrogate_set_sample(sesw_ctx *c, int64_t index, const double *eta, const double *U, const double *R,
                              const double *d_umean, const double *d_uM, const double *d_etabar, int where)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (index < 0 || index >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
    if (!eta || !U || !R || !d_umean || !d_uM || !d_etabar) return sesw::ctx_fail(c, SESW_EINVAL, "NULL sample array");
    const double *p[6] = {eta, U, R, d_umean, d_uM, d_etabar};
    const size_t n[6] = {(size_t)S.V, 2 * (size_t)S.E, 2 * (size_t)S.E, 2 * (size_t)S.E, 2 * (size_t)S.E, (size_t)S.V};
    const double *dp[6];
    if (where == SESW_HOST) {
        size_t o = 0;
        for (int k = 0; k < 6; k++) {
            SCK(cudaMemcpyAsync(S.stage + o, p[k], sizeof(double) * n[k], cudaMemcpyHostToDevice, c->stream));
            dp[k] = S.stage + o;
            o += n[k];
        }
    } else if (where == SESW_DEVICE) {
        for (int k = 0; k < 6; k++) dp[k] = p[k];
    } else {
        return sesw::ctx_fail(c, SESW_EINVAL, "where must be SESW_HOST or SESW_DEVICE");
    }
    sesw::k_sample_from_caller<<<sesw::grid1(std::max(S.V, S.E)), 256, 0, c->stream>>>(
        S.V, S.E, c->dm.vperm, c->dm.eperm, dp[0], dp[1], dp[2], dp[3], dp[4], dp[5], S.d_eta + (size_t)index * S.V,
        S.d_U + (size_t)index * 2 * S.E, S.d_R + (size_t)index * 2 * S.E, S.d_te + (size_t)index * 4 * S.E,
        S.d_tv + (size_t)index * S.V);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(c->stream));
    return SESW_OK;
}

int sesw_surrogate_record_input(sesw_ctx *c, int64_t index)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (index < 0 || index >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
    sesw::k_take_state<<<sesw::grid1(std::max(S.V, S.E)), 256, 0, c->stream>>>(
        S.V, S.E, c->ds.eta[c->parity], c->ds.U, c->ds.R, S.eslot, S.d_eta + (size_t)index * S.V,
        S.d_U + (size_t)index * 2 * S.E, S.d_R + (size_t)index * 2 * S.E);
    SCK(cudaGetLastError());
    return SESW_OK;
}

int sesw_surrogate_record_target(sesw_ctx *c, int64_t index)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (index < 0 || index >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
    if (!c->ds.eta_sum) return sesw::ctx_fail(c, SESW_ESTATE, "enable the step-mean elevation (sesw_set_eta_mean)");
    sesw::k_take_targets<<<sesw::grid1(std::max(S.V, S.E)), 256, 0, c->stream>>>(
        S.V, S.E, c->ds.eta_sum, c->args.inv_M, c->ds.U, c->ds.Umean, S.eslot, S.d_eta + (size_t)index * S.V,
        S.d_U + (size_t)index * 2 * S.E, S.d_te + (size_t)index * 4 * S.E, S.d_tv + (size_t)index * S.V);
    SCK(cudaGetLastError());
    return SESW_OK;
}

int sesw_surrogate_fit_scales(sesw_ctx *c, int64_t nsamples, double length_scale)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (nsamples < 1 || nsamples > S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "nsamples out of range");
    if (!c->have_params) return sesw::ctx_fail(c, SESW_ESTATE, "set parameters first");
    const int nb = 152 * 4;
    std::vector<double> acc(5, 0.0), h(8 * nb);
    for (long i = 0; i < nsamples; i++) {
        sesw::k_sumsq<<<nb, 256, 0, c->stream>>>(S.V, S.E, S.d_eta + (size_t)i * S.V, S.d_U + (size_t)i * 2 * S.E,
                                                 S.d_R + (size_t)i * 2 * S.E, S.d_te + (size_t)i * 4 * S.E,
                                                 S.d_tv + (size_t)i * S.V, S.red + 16);
        SCK(cudaMemcpyAsync(h.data(), S.red + 16, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
        for (int b = 0; b < nb; b++)
            for (int q = 0; q < 5; q++) acc[q] += h[8 * b + q];
    }
    auto rms = [&](double s, double n) { double r = sqrt(s / n); return r > 0.0 ? r : 1.0; };
    // H and f scales from the mesh (host copies are not kept: use the device maxima)
    std::vector<float> eH0(S.E), ef(S.E);
    SCK(cudaMemcpyAsync(eH0.data(), S.eH0, sizeof(float) * S.E, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaMemcpyAsync(ef.data(), S.ef, sizeof(float) * S.E, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    double hmax = 0.0, fmax = 0.0;
    for (int e = 0; e < S.E; e++) {
        hmax = std::max(hmax, (double)fabsf(eH0[e]));
        fmax = std::max(fmax, (double)fabsf(ef[e]));
    }
    double sc[sesw::NSCALE];
    sc[sesw::S_ETA] = rms(acc[0], (double)nsamples * S.V);
    sc[sesw::S_H] = hmax > 0.0 ? hmax : 1.0;
    sc[sesw::S_U] = rms(acc[1], (double)nsamples * 2 * S.E);
    sc[sesw::S_R] = rms(acc[2], (double)nsamples * 2 * S.E);
    sc[sesw::S_F] = fmax > 0.0 ? fmax : 1.0;
    sc[sesw::S_L] = length_scale > 0.0 ? length_scale : 1.0;
    sc[sesw::S_OU] = rms(acc[3], (double)nsamples * 4 * S.E);
    sc[sesw::S_OETA] = rms(acc[4], (double)nsamples * S.V);
    return sesw_surrogate_scales(c, nullptr, sc);
}

static int run_sample(sesw_ctx *c, long i, bool grad, bool adam, double *loss)
{
    Surrogate &S = *c->sur;
    sesw::features_of(S, c, i);
    SCK(sesw::forward(S, c->stream));
    SCK(sesw::loss_of(S, c, i, grad, S.red));
    if (grad) {
        SCK(sesw::backward(S, c->stream));
        if (adam) {
            S.adam_t++;
            const float c1 = (float)(1.0 / (1.0 - pow(S.b1, (double)S.adam_t)));
            const float c2 = (float)(1.0 / (1.0 - pow(S.b2, (double)S.adam_t)));
            sesw::k_adam<<<sesw::grid1(S.nparam), 256, 0, c->stream>>>(S.nparam, S.w32, S.w16, S.grad, S.am, S.av,
                                                                       (float)S.lr, (float)S.b1, (float)S.b2,
                                                                       (float)S.eps, c1, c2);
            SCK(cudaGetLastError());
            SCK(sesw::pack_tc(S, c->stream));
        }
    }
    if (loss) {
        double l = 0.0;
        SCK(cudaMemcpyAsync(&l, S.red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
        *loss = l;
    }
    return SESW_OK;
}

int sesw_surrogate_train(sesw_ctx *c, const int64_t *indices, int32_t n, double learning_rate, double *mean_loss)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (!indices || n < 1) return sesw::ctx_fail(c, SESW_EINVAL, "need at least one sample index");
    if (!(learning_rate > 0.0)) return sesw::ctx_fail(c, SESW_EINVAL, "learning rate must be positive");
    S.lr = learning_rate;
    double sum = 0.0;
    for (int k = 0; k < n; k++) {
        if (indices[k] < 0 || indices[k] >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
        double l = 0.0;
        STRY(run_sample(c, indices[k], true, true, mean_loss ? &l : nullptr));
        sum += l;
    }
    if (mean_loss) *mean_loss = sum / n;
    return SESW_OK;
}

int sesw_surrogate_loss(sesw_ctx *c, const int64_t *indices, int32_t n, double *mean_loss)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (!indices || n < 1 || !mean_loss) return sesw::ctx_fail(c, SESW_EINVAL, "need sample indices and an output");
    double sum = 0.0;
    for (int k = 0; k < n; k++) {
        if (indices[k] < 0 || indices[k] >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
        double l = 0.0;
        STRY(run_sample(c, indices[k], false, false, &l));
        sum += l;
    }
    *mean_loss = sum / n;
    return SESW_OK;
}

int sesw_surrogate_gradient(sesw_ctx *c, int64_t index, float *grad, double *loss)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (index < 0 || index >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
    STRY(run_sample(c, index, true, false, loss));
    if (grad) {
        SCK(cudaMemcpyAsync(grad, S.grad, sizeof(float) * S.nparam, cudaMemcpyDeviceToHost, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
    }
    return SESW_OK;
}

int sesw_surrogate_predict(sesw_ctx *c, int64_t index, double *out_e, double *out_v)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (index < 0 || index >= S.cap) return sesw::ctx_fail(c, SESW_EINVAL, "sample index out of range");
    STRY(run_sample(c, index, false, false, nullptr));
    std::vector<float> oe(4 * (size_t)S.E), ov(S.V);
    std::vector<int> vperm(S.V), eperm(S.E);
    SCK(cudaMemcpyAsync(oe.data(), S.oe, sizeof(float) * oe.size(), cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaMemcpyAsync(ov.data(), S.ov, sizeof(float) * ov.size(), cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaMemcpyAsync(vperm.data(), c->dm.vperm, sizeof(int) * S.V, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaMemcpyAsync(eperm.data(), c->dm.eperm, sizeof(int) * S.E, cudaMemcpyDeviceToHost, c->stream));
    SCK(cudaStreamSynchronize(c->stream));
    for (int e = 0; e < S.E; e++)
        for (int q = 0; q < 4; q++) out_e[4 * (size_t)eperm[e] + q] = oe[4 * (size_t)e + q];
    for (int v = 0; v < S.V; v++) out_v[vperm[v]] = ov[v];
    return SESW_OK;
}

int sesw_surrogate_advance(sesw_ctx *c, int32_t nsteps, double resid_tol, int32_t *n_fallback, double *last_resid)
{
    STRY(need_sur(c));
    Surrogate &S = *c->sur;
    if (!c->have_params) return sesw::ctx_fail(c, SESW_ESTATE, "set parameters first");
    if (c->params.scheme != 0) return sesw::ctx_fail(c, SESW_EINVAL, "the surrogate replaces the SE subcycle");
    if (c->visc_on || c->have_W)
        return sesw::ctx_fail(c, SESW_EINVAL,
                              "the surrogate is trained without the barotropic viscosity and the freshwater flux");
    int fb = 0;
    double resid = 0.0;
    const float tau = (float)c->params.tau;
    const int nb = 152 * 4;
    for (int n = 0; n < nsteps; n++) {
        float *eta0 = c->ds.eta[c->parity];
        // the current state as network input, and a copy for the fallback
        sesw::k_take_state<<<sesw::grid1(std::max(S.V, S.E)), 256, 0, c->stream>>>(
            S.V, S.E, eta0, c->ds.U, c->ds.R, S.eslot, S.cur_eta, S.cur_U, S.cur_R);
        SCK(cudaMemcpyAsync(S.save_eta, eta0, sizeof(float) * S.V, cudaMemcpyDeviceToDevice, c->stream));
        SCK(cudaMemcpyAsync(S.save_U, c->ds.U, sizeof(float2) * c->dm.nslot, cudaMemcpyDeviceToDevice, c->stream));
        sesw::k_features<<<sesw::grid1(std::max(S.V, S.E)), 256, 0, c->stream>>>(
            S.V, S.E, S.cur_eta, S.cur_U, S.cur_R, c->dm.h0_v, S.eH0, S.ef, S.scales, S.xv, S.xe);
        SCK(sesw::forward(S, c->stream, false));
        sesw::k_apply_elems<<<sesw::grid1(c->dm.nslot), 256, 0, c->stream>>>(S.E, c->dm.nslot, c->dm.slot_v, S.oe,
                                                                              S.scales, S.cur_U, c->ds.U, c->ds.Umean);
        float *eta1 = c->ds.eta[c->parity ^ 1];
        sesw::k_apply_verts<<<sesw::grid1(S.V), 256, 0, c->stream>>>(S.V, S.voff, S.vinc, S.egrad, S.earea,
                                                                      c->dm.inv_av, c->ds.Umean, S.ov, S.scales, tau,
                                                                      eta0, eta1, S.etabar);
        sesw::k_residual<<<nb, 256, 0, c->stream>>>(S.E, S.etri, S.egrad, S.earea, S.eH0, S.ef, S.eslot, c->ds.U,
                                                    c->ds.Umean, S.cur_U, S.cur_R, S.etabar, tau, c->args.g,
                                                    c->args.theta, (float)c->params.M, c->params.nonlinear_h,
                                                    S.red + 16);
        SCK(cudaGetLastError());
        std::vector<double> h(2 * nb);
        SCK(cudaMemcpyAsync(h.data(), S.red + 16, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nb; k++) {
            a += h[2 * k];
            b += h[2 * k + 1];
        }
        resid = sqrt(a / (b + 1e-300));
        if (resid <= resid_tol && std::isfinite(resid)) {
            c->parity ^= 1;
        } else {
            // the plain subcycle takes this step instead
            SCK(cudaMemcpyAsync(eta0, S.save_eta, sizeof(float) * S.V, cudaMemcpyDeviceToDevice, c->stream));
            SCK(cudaMemcpyAsync(c->ds.U, S.save_U, sizeof(float2) * c->dm.nslot, cudaMemcpyDeviceToDevice, c->stream));
            STRY(sesw::ctx_enqueue_step(c));
            fb++;
        }
    }
    if (n_fallback) *n_fallback = fb;
    if (last_resid) *last_resid = resid;
    return SESW_OK;
}

}  // extern "C"
