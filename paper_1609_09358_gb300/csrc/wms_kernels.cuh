// wms_kernels.cuh -- training kernels of the learned weighted min-sum BP: forward with stored
// messages and the hand-written reverse sweep that returns the gradient of the per-edge,
// per-iteration scale factors.
//
// Forward (T iterations, no early stop): the BP of Sec. II-B with every g term scaled,
//   R sweep, PE stage s:  R[s+1][j]   = clip(w[t][0][s-1][j]   g(R[s][j], L'[s+1][j+d] + R[s][j+d]))
//                         R[s+1][j+d] = clip(w[t][0][s-1][j+d] g(R[s][j], L'[s+1][j]) + R[s][j+d])
//   L sweep, PE stage s:  L[s][j]     = clip(w[t][1][s-1][j]   g(L[s+1][j], L[s+1][j+d] + R[s][j+d]))
//                         L[s][j+d]   = clip(w[t][1][s-1][j+d] g(R[s][j], L[s+1][j]) + L[s+1][j+d])
// (L' = previous iteration), output LLR(u) = L[1] + R[1] of the last iteration, or of every
// iteration (`all`: a per-iteration training loss).  Same arithmetic, operation by operation,
// as the inference kernel with weights, so both agree bit for bit.
//
// Backward: reverse-mode through the unrolled iterations.  Message versions: R^t[s+1] depends on
// R^t[s] and L^{t-1}[s+1]; L^t[s] on L^t[s+1] and R^t[s].  Reverse order: for t = T-1..0 the L
// sweep is undone for s = 1..n, then the R sweep for s = n..1; by then every consumer of a message
// has been undone, so its adjoint is complete.  Within a stage each input node feeds exactly one PE,
// so adjoints accumulate without atomics; the weight gradients of all frames are summed with
// atomicAdd.  Subgradients: g(a, b) = sign(a) sign(b) min(|a|, |b|) passes the adjoint times
// sign(b) to a when |a| <= |b| and times sign(a) to b otherwise; clip passes it where |x| < M.
//
// Layout: one CTA of N/2 threads per frame, thread p owns the PE of its stage.  Per frame the
// workspace holds the stored messages [2][T][n][N] (R columns 2..n+1, L columns 1..n) and the
// adjoints [3][n+2][N] (current R, current L, previous-iteration L).
#pragma once

#include "polar_common.cuh"

namespace polar {

struct WMSArgs {
    const float* llr;
    int B, T;
    float M;
    const float* w;        // [T][2][n][N]
    int all;               // outputs / their adjoints for every iteration ([T][B][N]) or the last ([B][N])
    float* llr_u;          // forward output
    const float* grad_u;   // backward input, same shape as llr_u
    float* grad_w;         // backward output [T][2][n][N], accumulated
    float* store;          // [B][2][T][n][N]
    float* adj;            // [B][3][n+2][N]
    const DevCode* code;
};

__device__ __forceinline__ size_t wms_store_frame(int T, int n, int N) { return (size_t)2 * T * n * N; }
__device__ __forceinline__ float wms_sgn(float v) { return v < 0.0f ? -1.0f : 1.0f; }

// node pair of PE p at stage s (bit s-1 of j clear)
__device__ __forceinline__ int pe_node(int p, int s) { return ((p >> (s - 1)) << s) | (p & ((1 << (s - 1)) - 1)); }

__global__ void __launch_bounds__(1024) wms_forward_kernel(const WMSArgs a)
{
    const DevCode& C = *a.code;
    const int N = C.N, n = C.n, T = a.T;
    const int b = blockIdx.x, p = threadIdx.x;
    const float M = a.M;
    const float* y = a.llr + (size_t)b * N;
    float* Rst = a.store + (size_t)b * wms_store_frame(T, n, N);
    float* Lst = Rst + (size_t)T * n * N;
    auto Rcol = [&](int t, int c) -> float* { return Rst + ((size_t)t * n + (c - 2)) * N; };  // c = 2..n+1
    auto Lcol = [&](int t, int c) -> float* { return Lst + ((size_t)t * n + (c - 1)) * N; };  // c = 1..n
    auto R1 = [&](int i) -> float { return frozen_at(C.frozen_bits, i) ? M : 0.0f; };
    auto ch = [&](int i) -> float { return stage_clip(y[i], M); };
    auto W = [&](int t, int dir, int s, int i) -> float { return a.w[(((size_t)t * 2 + dir) * n + (s - 1)) * N + i]; };
    for (int t = 0; t < T; ++t) {
        for (int s = 1; s <= n; ++s) {
            const int j = pe_node(p, s), jd = j + (1 << (s - 1));
            const float a1 = s == 1 ? R1(j) : Rcol(t, s)[j];
            const float a2 = s == 1 ? R1(jd) : Rcol(t, s)[jd];
            float l1 = 0.0f, l2 = 0.0f;
            if (s + 1 == n + 1) {
                l1 = ch(j);
                l2 = ch(jd);
            } else if (t > 0) {
                l1 = Lcol(t - 1, s + 1)[j];
                l2 = Lcol(t - 1, s + 1)[jd];
            }
            const float o1 = clipm(fmul(W(t, 0, s, j), xmin(a1, fadd(l2, a2))), M);
            const float o2 = clipm(fadd(fmul(W(t, 0, s, jd), xmin(a1, l1)), a2), M);
            Rcol(t, s + 1)[j] = o1;
            Rcol(t, s + 1)[jd] = o2;
            __syncthreads();
        }
        for (int s = n; s >= 1; --s) {
            const int j = pe_node(p, s), jd = j + (1 << (s - 1));
            const float a1 = s == 1 ? R1(j) : Rcol(t, s)[j];
            const float a2 = s == 1 ? R1(jd) : Rcol(t, s)[jd];
            const float l1 = s == n ? ch(j) : Lcol(t, s + 1)[j];
            const float l2 = s == n ? ch(jd) : Lcol(t, s + 1)[jd];
            const float o1 = clipm(fmul(W(t, 1, s, j), xmin(l1, fadd(l2, a2))), M);
            const float o2 = clipm(fadd(fmul(W(t, 1, s, jd), xmin(a1, l1)), l2), M);
            Lcol(t, s)[j] = o1;
            Lcol(t, s)[jd] = o2;
            __syncthreads();
        }
        if (a.all || t == T - 1) {
            float* out = a.llr_u + ((size_t)(a.all ? t : 0) * a.B + b) * N;
            for (int i = p; i < N; i += blockDim.x) out[i] = fadd(Lcol(t, 1)[i], R1(i));
        }
    }
}

// Reverse of one PE: forward o1 = clip(w1 g(u, v + q)), o2 = clip(w2 g(r, u) + q2) in the
// generic form shared by both sweeps; returns adjoints of the inputs and the weight gradients.
struct PEGrad {
    float du, dv, dq, dr, dq2, dw1, dw2;
};
__device__ __forceinline__ PEGrad pe_backward(float u, float v, float q, float r, float q2, float w1, float w2, float M,
                                              float go1, float go2)
{
    // o1 = clip(w1 * g(u, v + q)); o2 = clip(w2 * g(r, u) + q2)
    PEGrad G{0, 0, 0, 0, 0, 0, 0};
    const float s1 = fadd(v, q);
    const float g1 = xmin(u, s1);
    const float x1 = fmul(w1, g1);
    const float g2 = xmin(r, u);
    const float x2 = fadd(fmul(w2, g2), q2);
    const float c1 = fabsf(x1) < M ? go1 : 0.0f;
    const float c2 = fabsf(x2) < M ? go2 : 0.0f;
    G.dw1 = c1 * g1;
    G.dw2 = c2 * g2;
    const float gg1 = c1 * w1, gg2 = c2 * w2;
    G.dq2 = c2;
    if (fabsf(u) <= fabsf(s1)) {
        G.du += gg1 * wms_sgn(s1);
    } else {
        const float d = gg1 * wms_sgn(u);
        G.dv += d;
        G.dq += d;
    }
    if (fabsf(r) <= fabsf(u))
        G.dr += gg2 * wms_sgn(u);
    else
        G.du += gg2 * wms_sgn(r);
    return G;
}

__global__ void __launch_bounds__(1024) wms_backward_kernel(const WMSArgs a)
{
    const DevCode& C = *a.code;
    const int N = C.N, n = C.n, T = a.T;
    const int b = blockIdx.x, p = threadIdx.x;
    const float M = a.M;
    const float* y = a.llr + (size_t)b * N;
    const float* Rst = a.store + (size_t)b * wms_store_frame(T, n, N);
    const float* Lst = Rst + (size_t)T * n * N;
    auto Rcol = [&](int t, int c) -> const float* { return Rst + ((size_t)t * n + (c - 2)) * N; };
    auto Lcol = [&](int t, int c) -> const float* { return Lst + ((size_t)t * n + (c - 1)) * N; };
    auto R1 = [&](int i) -> float { return frozen_at(C.frozen_bits, i) ? M : 0.0f; };
    auto ch = [&](int i) -> float { return stage_clip(y[i], M); };
    auto W = [&](int t, int dir, int s, int i) -> float { return a.w[(((size_t)t * 2 + dir) * n + (s - 1)) * N + i]; };
    auto GW = [&](int t, int dir, int s, int i) -> float* { return a.grad_w + (((size_t)t * 2 + dir) * n + (s - 1)) * N + i; };
    float* adj = a.adj + (size_t)b * 3 * (n + 2) * N;
    float* aR = adj;  // [n+2][N], column c
    float* aLbuf[2] = {adj + (size_t)(n + 2) * N, adj + (size_t)2 * (n + 2) * N};
    for (size_t i = p; i < (size_t)3 * (n + 2) * N; i += blockDim.x) adj[i] = 0.0f;
    __syncthreads();
    for (int t = T - 1; t >= 0; --t) {
        float* aL = aLbuf[(T - 1 - t) & 1];       // adjoints of L^t
        float* aLp = aLbuf[(T - t) & 1];          // adjoints of L^{t-1}
        // LLR(u) of iteration t is L^t[1] + R[1]: its adjoint enters at column 1 (nothing else
        // reads L[1], so the column holds no other contribution)
        if (a.all || t == T - 1) {
            const float* gu = a.grad_u + ((size_t)(a.all ? t : 0) * a.B + b) * N;
            for (int i = p; i < N; i += blockDim.x) aL[1 * N + i] += gu[i];
            __syncthreads();
        }
        // ---- undo the L sweep: s = 1..n
        for (int s = 1; s <= n; ++s) {
            const int j = pe_node(p, s), jd = j + (1 << (s - 1));
            const float a1 = s == 1 ? R1(j) : Rcol(t, s)[j];
            const float a2 = s == 1 ? R1(jd) : Rcol(t, s)[jd];
            const float l1 = s == n ? ch(j) : Lcol(t, s + 1)[j];
            const float l2 = s == n ? ch(jd) : Lcol(t, s + 1)[jd];
            // o1 = clip(w1 g(l1, l2 + a2)), o2 = clip(w2 g(a1, l1) + l2)
            const PEGrad G = pe_backward(l1, l2, a2, a1, l2, W(t, 1, s, j), W(t, 1, s, jd), M, aL[s * N + j],
                                         aL[s * N + jd]);
            atomicAdd(GW(t, 1, s, j), G.dw1);
            atomicAdd(GW(t, 1, s, jd), G.dw2);
            if (s < n) {
                aL[(s + 1) * N + j] += G.du;
                aL[(s + 1) * N + jd] += G.dv + G.dq2;
            }
            if (s > 1) {
                aR[s * N + j] += G.dr;
                aR[s * N + jd] += G.dq;
            }
            __syncthreads();
        }
        // ---- undo the R sweep: s = n..1
        for (int s = n; s >= 1; --s) {
            const int j = pe_node(p, s), jd = j + (1 << (s - 1));
            const float a1 = s == 1 ? R1(j) : Rcol(t, s)[j];
            const float a2 = s == 1 ? R1(jd) : Rcol(t, s)[jd];
            float l1 = 0.0f, l2 = 0.0f;
            if (s == n) {
                l1 = ch(j);
                l2 = ch(jd);
            } else if (t > 0) {
                l1 = Lcol(t - 1, s + 1)[j];
                l2 = Lcol(t - 1, s + 1)[jd];
            }
            // o1 = clip(w1 g(a1, l2 + a2)), o2 = clip(w2 g(a1, l1) + a2): generic form with
            // u = a1, v = l2, q = a2, r = l1 (g(r, u) = g(l1, a1) = g(a1, l1)), q2 = a2
            const PEGrad G = pe_backward(a1, l2, a2, l1, a2, W(t, 0, s, j), W(t, 0, s, jd), M, aR[(s + 1) * N + j],
                                         aR[(s + 1) * N + jd]);
            atomicAdd(GW(t, 0, s, j), G.dw1);
            atomicAdd(GW(t, 0, s, jd), G.dw2);
            if (s > 1) {
                aR[s * N + j] += G.du;
                aR[s * N + jd] += G.dq + G.dq2;
            }
            if (s < n && t > 0) {
                aLp[(s + 1) * N + j] += G.dr;
                aLp[(s + 1) * N + jd] += G.dv;
            }
            __syncthreads();
        }
        // the adjoints of this iteration are consumed: clear them for iteration t-2 / t-1
        for (int i = p; i < (n + 2) * N; i += blockDim.x) {
            aL[i] = 0.0f;
            aR[i] = 0.0f;
        }
        __syncthreads();
    }
}

}  // namespace polar
