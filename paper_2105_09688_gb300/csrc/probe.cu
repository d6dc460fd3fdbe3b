// probe.cu -- ssm_pipe_probe: measured throughput of the FP32 pipes the pair sums run
// on (no counterpart in the paper).  The pair kernels are bound by the FP32 FMA pipe
// and the special-function unit (MUFU), whose nominal rates are not what a sustained
// stream of packed FFMA2 or of MUFU.RCP reaches; this probe measures them on the
// current device so that roofline fractions can be read against measured rates.
//
// Every thread runs eight independent dependency chains of one instruction kind in
// registers for `iters` iterations and writes one float (so nothing is optimised
// away); the grid is eight 256-thread blocks per SM.  Block 0 reads clock64 and the
// global nanosecond timer around its work, which gives the SM clock; the rate is
// lane operations per clock per SM = lanes x ops / (elapsed ns x GHz x SMs).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ssm.h"
#include "ssm_device.cuh"

namespace {

enum : int { PR_FFMA = 0, PR_FFMA2 = 1, PR_RCP = 2, PR_EX2 = 3, PR_N = 4 };

template <int OP>
__global__ void __launch_bounds__(256) k_pipe_probe(float *out, int iters, unsigned long long *clk) {
    unsigned long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    float v[8];
    float2 p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i] = 0.5f + 1e-4f * (float)(threadIdx.x & 63) + 0.01f * (float)i;
        p[i] = make_float2(v[i], v[i] + 0.1f);
    }
    const float2 m2 = make_float2(0.999f, 0.998f), a2 = make_float2(1e-3f, 2e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == PR_FFMA) v[i] = fmaf(v[i], 0.999f, 1e-3f);
            if (OP == PR_FFMA2) p[i] = __ffma2_rn(p[i], m2, a2);
            if (OP == PR_RCP) v[i] = ssm::rcp_approx(v[i]) + 0.25f;     // stays in [1.25, 4.25]
            if (OP == PR_EX2) v[i] = ssm::ex2_approx(-v[i]);             // stays in (0.5, 1)
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += v[i] + p[i].x + p[i].y;
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long c1 = clock64(), t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
}

template <int OP>
cudaError_t run_probe(int sms, float *out, unsigned long long *dclk, int iters, double lane_ops, double *rate,
                      double *ghz) {
    const int blocks = sms * 8, threads = 256;
    k_pipe_probe<OP><<<blocks, threads>>>(out, 64, dclk);   // warm-up
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
        k_pipe_probe<OP><<<blocks, threads>>>(out, iters, dclk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long hclk[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(hclk, dclk, sizeof hclk, cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double g = hclk[1] > 0 ? (double)hclk[0] / (double)hclk[1] : 0.0;
    const double ops = (double)blocks * threads * iters * lane_ops;
    *ghz = g;
    *rate = (g > 0.0 && ms > 0.f) ? ops / ((double)ms * 1e-3) / (g * 1e9) / sms : 0.0;
    return cudaSuccess;
}

}  // namespace

extern "C" ssm_status ssm_pipe_probe(double *out) {
    if (!out) return SSM_EINVAL;
    const int sms = ssm::device_sms();
    if (sms <= 0) return SSM_ECUDA;
    float *buf = nullptr;
    unsigned long long *dclk = nullptr;
    cudaError_t e = cudaMalloc((void **)&buf, sizeof(float) * (size_t)sms * 8 * 256);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dclk, 2 * sizeof(unsigned long long));
    double ghz[PR_N] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = run_probe<PR_FFMA>(sms, buf, dclk, 8192, 8.0, &out[0], &ghz[0]);
    if (e == cudaSuccess) e = run_probe<PR_FFMA2>(sms, buf, dclk, 8192, 16.0, &out[1], &ghz[1]);
    if (e == cudaSuccess) e = run_probe<PR_RCP>(sms, buf, dclk, 2048, 8.0, &out[2], &ghz[2]);
    if (e == cudaSuccess) e = run_probe<PR_EX2>(sms, buf, dclk, 4096, 8.0, &out[3], &ghz[3]);
    if (e == cudaSuccess) out[4] = (ghz[0] + ghz[1] + ghz[2] + ghz[3]) / 4.0;
    cudaFree(buf);
    cudaFree(dclk);
    return e == cudaSuccess ? SSM_OK : SSM_ECUDA;
}
