// The adjoint of the loss: dL/dx_i along the chosen neighbours (derivative of Eq. 1 / Eq. 2)
// scattered to the picked face's vertices with the barycentric weights (Eq. 4).
#include "dc_internal.cuh"

namespace dc {

namespace {

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, DC_OK, code); }

constexpr int BWD_THREADS = 512;

// G[v_c] += w_c * g for the three vertices of face f (indices were validated when sampling)
__device__ __forceinline__ void scatter(float* __restrict__ G, const int* __restrict__ faces,
                                        int V, int4 q, float gx, float gy, float gz) {
    const int f = q.x;
    const float wc[3] = {__int_as_float(q.y), __int_as_float(q.z), __int_as_float(q.w)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int v = faces[3 * f + c];
        if ((unsigned)v >= (unsigned)V) continue;
        atomicAdd(&G[3 * v + 0], __fmul_rn(wc[c], gx));
        atomicAdd(&G[3 * v + 1], __fmul_rn(wc[c], gy));
        atomicAdd(&G[3 * v + 2], __fmul_rn(wc[c], gz));
    }
}

// One CTA per frame; the frame's V x 3 accumulator lives in shared memory when it fits
// (use_smem), else the CTA zeroes and accumulates into the output directly.
__global__ void __launch_bounds__(BWD_THREADS) k_bwd(Ws w, int bidir, int use_smem) {
    extern __shared__ float s_acc[];
    const FrameDesc* fr = w.frames + blockIdx.x;
    float* out = fr->grad;
    if (!out || !fr->verts) return;
    const int V = fr->V, N = fr->N, M = fr->M, row0 = fr->row0;
    const int* faces = fr->faces;
    const float* tgt = fr->tgt;
    float* G = use_smem ? s_acc : out;
    for (int v = threadIdx.x; v < 3 * V; v += BWD_THREADS) G[v] = 0.0f;
    __syncthreads();

    const float cab = bidir ? __fdiv_rn(__fmul_rn(2.0f, fr->gscale), (float)N)
                            : __fmul_rn(2.0f, fr->gscale);
    const float cba = __fdiv_rn(__fmul_rn(2.0f, fr->gscale), (float)M);

    // sim -> target term of every sampled point
    for (int i = threadIdx.x; i < N; i += BWD_THREADS) {
        const int j = fr->nn_ab[i];
        const int4 q = w.fw[row0 + i];
        if ((unsigned)j >= (unsigned)M || q.x < 0) {
            set_status(&w.hdr->status, DC_EINVAL);
            continue;
        }
        const float4 x = w.x[row0 + i];
        const float* y = tgt + 3LL * j;
        scatter(G, faces, V, q, __fmul_rn(cab, __fsub_rn(x.x, y[0])),
                __fmul_rn(cab, __fsub_rn(x.y, y[1])), __fmul_rn(cab, __fsub_rn(x.z, y[2])));
    }
    // target -> sim term, routed to the face of the target's nearest sampled point
    if (bidir) {
        for (int j = threadIdx.x; j < M; j += BWD_THREADS) {
            const int i = fr->nn_ba[j];
            if ((unsigned)i >= (unsigned)N) {
                set_status(&w.hdr->status, DC_EINVAL);
                continue;
            }
            const int4 q = w.fw[row0 + i];
            if (q.x < 0) continue;
            const float4 x = w.x[row0 + i];
            const float* y = tgt + 3LL * j;
            scatter(G, faces, V, q, __fmul_rn(cba, __fsub_rn(x.x, y[0])),
                    __fmul_rn(cba, __fsub_rn(x.y, y[1])), __fmul_rn(cba, __fsub_rn(x.z, y[2])));
        }
    }
    if (use_smem) {
        __syncthreads();
        for (int v = threadIdx.x; v < 3 * V; v += BWD_THREADS) out[v] = s_acc[v];
    }
}

// ---- gradient with respect to given sim points (dc_chamfer_bwd) ----
__global__ void __launch_bounds__(256) k_cbwd_rows(const float* a, const float* b,
                                                   const int* nn_ab, int T, int N, int M,
                                                   int bidir, const float* g, float* grad) {
    const long long n = (long long)T * N;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const int t = (int)(e / N);
        const int j = nn_ab[e];
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if ((unsigned)j < (unsigned)M) {
            const float c = bidir ? __fdiv_rn(__fmul_rn(2.0f, g[t]), (float)N)
                                  : __fmul_rn(2.0f, g[t]);
            const float* y = b + 3LL * ((long long)t * M + j);
            gx = __fmul_rn(c, __fsub_rn(a[3 * e], y[0]));
            gy = __fmul_rn(c, __fsub_rn(a[3 * e + 1], y[1]));
            gz = __fmul_rn(c, __fsub_rn(a[3 * e + 2], y[2]));
        }
        grad[3 * e] = gx;
        grad[3 * e + 1] = gy;
        grad[3 * e + 2] = gz;
    }
}

__global__ void __launch_bounds__(256) k_cbwd_cols(const float* a, const float* b,
                                                   const int* nn_ba, int T, int N, int M,
                                                   const float* g, float* grad) {
    const long long n = (long long)T * M;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const int t = (int)(e / M);
        const int i = nn_ba[e];
        if ((unsigned)i >= (unsigned)N) continue;
        const float c = __fdiv_rn(__fmul_rn(2.0f, g[t]), (float)M);
        const long long ia = (long long)t * N + i;
        const float* x = a + 3 * ia;
        atomicAdd(&grad[3 * ia], __fmul_rn(c, __fsub_rn(x[0], b[3 * e])));
        atomicAdd(&grad[3 * ia + 1], __fmul_rn(c, __fsub_rn(x[1], b[3 * e + 1])));
        atomicAdd(&grad[3 * ia + 2], __fmul_rn(c, __fsub_rn(x[2], b[3 * e + 2])));
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

int g_smem_limit[64];

}  // namespace

cudaError_t launch_bwd(const Ws& w, int n_frames, int max_v, int mode, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_smem_limit[dev] == 0) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (optin <= 0) optin = 48 * 1024;
        cudaError_t e = cudaFuncSetAttribute(k_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             optin);
        if (e != cudaSuccess) return e;
        g_smem_limit[dev] = optin;
    }
    const size_t need = (size_t)max_v * 3 * sizeof(float);
    const int use_smem = need <= (size_t)g_smem_limit[dev];
    k_bwd<<<n_frames, BWD_THREADS, use_smem ? need : 0, s>>>(w, mode == DC_BIDIR_MEAN, use_smem);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_chamfer_bwd_points(const float* a, const float* b, const int* nn_ab,
                                      const int* nn_ba, int T, int N, int M, int mode,
                                      const float* g, float* grad_a, cudaStream_t s) {
    const int bidir = mode == DC_BIDIR_MEAN;
    k_cbwd_rows<<<grid_for((long long)T * N, 256), 256, 0, s>>>(a, b, nn_ab, T, N, M, bidir, g,
                                                                 grad_a);
    count_launch();
    if (bidir) {
        k_cbwd_cols<<<grid_for((long long)T * M, 256), 256, 0, s>>>(a, b, nn_ba, T, N, M, g,
                                                                     grad_a);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace dc
