// Host-side prototypes shared by the kernel launchers and the C ABI.
#pragma once

#include "ccfr_device.cuh"

namespace ccfr {

// Stage boundaries recorded by ccfr_step_timed (CUDA events on the launch stream).
enum Stage {
    ST_PREDICT = 0, ST_GRID_EXTENT, ST_GRID_COUNT, ST_GRID_SCAN, ST_GRID_SCATTER,
    ST_EMIT_VF, ST_EMIT_EE, ST_EMIT_PP, ST_XPBD, ST_PROJECT, ST_MISC, ST_GRID_UNITS, ST_EMIT_VF_BIG,
    ST_EMIT_EE_BIG, ST_PROJECT_HEAVY, ST_PROJECT_SHORT, ST_RESPONSE, N_STAGES
};

struct StageTimer {
    cudaEvent_t* ev;      // pool
    int* stage;           // stage of the interval that ends at event i
    int n, cap;
    void mark(int s, cudaStream_t st) {
        if (n < cap) { cudaEventRecord(ev[n], st); stage[n] = s; ++n; }
    }
};

struct PairOutHost {
    int* out[3];
    long cap[3];
    unsigned long long* count;   // device [3]
};

// A second stream of a context with two events: the region build forks the
// edge-edge and point-point emission onto it, so that they run beside the
// vertex-face and oversized-primitive emission (graph branches under stream
// capture), and joins it back before the region is used.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

void launch_build(const DevCtx& c, const float4* x, cudaStream_t st, int mode, const PairOutHost* po,
                  unsigned* tile_sums, int n_buckets_total, StageTimer* tm = nullptr,
                  const SideStream* side = nullptr);
cudaError_t configure_kernels();
void launch_clear_regions(const DevCtx& c, cudaStream_t st);
void launch_project(const DevCtx& c, const float4* xb, float4* xio, unsigned char* halt, cudaStream_t st);
void launch_predict(const DevCtx& c, const float4* x, const float4* v, cudaStream_t st);
void launch_iteration(const DevCtx& c, float4* x, cudaStream_t st, const int* color_off, int n_colors,
                      unsigned* tile_sums, int n_buckets_total, int early_exit, StageTimer* tm = nullptr,
                      const SideStream* side = nullptr, const int* tcolor_off = nullptr, int n_tcolors = 0);
void launch_update(const DevCtx& c, const float4* x, float4* v, cudaStream_t st);
void launch_rest_state(const DevCtx& c, const float4* x, cudaStream_t st);
void launch_load_regions(const DevCtx& c, const float4* planes, const int* count, int cap, cudaStream_t st);
void launch_dmin_export(const DevCtx& c, float* out, cudaStream_t st);

}  // namespace ccfr
