// probe.cu -- the measured peak rate of the dominance test (Def. 1) on this
// GPU, the denominator of the grid-dominance kernel's roofline.
//
// Every thread keeps kProbeCands candidate rows in registers and tests each
// against a target cell [lo, hi] per attribute: s dominates the cell's corner
// when s_q <= hi_q for every attribute and s_q < lo_q for one, d "<=" and d
// "<" comparisons folded into one predicate -- the 2d compare lane-ops per
// test that the grid-dominance kernel counts as its algorithmic work. The
// cell moves every iteration, so no comparison can be hoisted out of the
// loop; the move costs 2d adds per kProbeCands tests. Operands never leave
// registers: the rate is bounded by the integer pipes alone.
//
// It also holds the check of the cooperative sorts' bounded grid-wide wait
// (gres_barrier_probe): one block stays away from the barrier on purpose, and
// the others must give up, flag the timeout and return.
#include "radix.cuh"

namespace gres {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCands = 16;

__device__ __forceinline__ uint32_t lcg(uint32_t &h) {
    h = h * 1664525u + 1013904223u;
    return h;
}

template <int D>
__global__ void __launch_bounds__(kProbeThreads) k_test_peak(uint32_t seed, int iters, unsigned long long *sink) {
    uint32_t h = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
    uint32_t s[kProbeCands][D];
    #pragma unroll
    for (int j = 0; j < kProbeCands; j++) {
        #pragma unroll
        for (int q = 0; q < D; q++) s[j][q] = lcg(h) >> 8;   // values below 2^24
    }
    uint32_t lo[D], hi[D];
    #pragma unroll
    for (int q = 0; q < D; q++) {
        lo[q] = lcg(h) >> 8;
        hi[q] = lo[q] + (1u << 20);
    }
    uint32_t hits = 0;
    for (int it = 0; it < iters; it++) {
        #pragma unroll
        for (int j = 0; j < kProbeCands; j++) {
            bool le = true, lt = false;
            #pragma unroll
            for (int q = 0; q < D; q++) {
                le &= s[j][q] <= hi[q];
                lt |= s[j][q] < lo[q];
            }
            hits += (le && lt) ? 1u : 0u;
        }
        #pragma unroll
        for (int q = 0; q < D; q++) {
            lo[q] += 0x00012345u + (uint32_t)q;
            hi[q] += 0x00012345u + (uint32_t)q;
        }
    }
    // hits <= iters * kProbeCands < 2^31: never true, but the compiler cannot know
    if (hits == 0xFFFFFFFFu) *sink = hits;
}

// blocks == 0: one full wave (resident blocks per SM x SMs).
template <int D>
cudaError_t launch_d(int iters, int blocks, unsigned long long *sink, cudaStream_t st, double *lane_ops) {
    if (blocks == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_test_peak<D>,
                                                                                kProbeThreads, 0);
        if (e != cudaSuccess) return e;
        blocks = (per_sm > 0 ? per_sm : 1) * sms;
    }
    *lane_ops = (double)blocks * kProbeThreads * (double)iters * kProbeCands * 2.0 * D;
    k_test_peak<D><<<blocks, kProbeThreads, 0, st>>>(0x2545F491u, iters, sink);
    note_launch();
    return cudaGetLastError();
}

// Every block but `absent` waits at one grid-wide barrier (words: arrivals,
// generation, status). With absent in [0, gridDim.x) the waits run out.
__global__ void __launch_bounds__(kRxThreads) k_barrier_probe(unsigned *words, int absent) {
    __shared__ int ok;
    if ((int)blockIdx.x == absent) return;
    grid_barrier(words, words + 2, &ok);
}

}  // namespace

cudaError_t launch_test_peak(int d, int iters, int blocks, unsigned long long *sink, cudaStream_t st,
                             double *lane_ops) {
    switch (d) {
        case 1: return launch_d<1>(iters, blocks, sink, st, lane_ops);
        case 2: return launch_d<2>(iters, blocks, sink, st, lane_ops);
        case 3: return launch_d<3>(iters, blocks, sink, st, lane_ops);
        case 4: return launch_d<4>(iters, blocks, sink, st, lane_ops);
        case 5: return launch_d<5>(iters, blocks, sink, st, lane_ops);
        case 6: return launch_d<6>(iters, blocks, sink, st, lane_ops);
        case 7: return launch_d<7>(iters, blocks, sink, st, lane_ops);
        default: return launch_d<8>(iters, blocks, sink, st, lane_ops);
    }
}

}  // namespace gres

extern "C" gres_status gres_barrier_probe(int32_t absent, unsigned *d_words, void *stream, uint32_t *h_status) {
    if (!d_words || !h_status) return gres::set_error(GRES_EINVAL, "d_words / h_status is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_words, 0, 3 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = gres::launch_coop(gres::k_barrier_probe, sms, st, d_words, (int)absent);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_status, d_words + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return gres::set_error(GRES_ECUDA, cudaGetErrorString(e));
    if (*h_status & gres::kStatusTimeout) return gres::set_error(GRES_ETIMEOUT, "a grid-wide wait ran out");
    return GRES_OK;
}
