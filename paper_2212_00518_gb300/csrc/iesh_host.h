// iesh_host.h -- host-side helpers shared by the library's contexts
// (internal): kernel timing with CUDA events and pointer classification.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/iesh.h"

namespace iesh {

// Per-class device time of bracketed launches.  With timing on, run()
// records an event pair around the launch on the given stream; fold()
// synchronises the last event and accumulates the elapsed times.  Event
// objects are recycled through a pool.
struct KernelTimer {
    bool on = false;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[IESH_K_COUNT] = {0};
    int64_t n[IESH_K_COUNT] = {0};

    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }

    cudaError_t fold()
    {
        if (recs.empty()) return cudaSuccess;
        cudaError_t err = cudaEventSynchronize(recs.back().b);
        for (auto &r : recs) {
            float m = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&m, r.a, r.b);
            ms[r.cls] += m;
            n[r.cls] += 1;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
        return err;
    }

    template <class Fn>
    cudaError_t run(cudaStream_t st, int cls, Fn fn)
    {
        if (!on) return fn();
        cudaEvent_t a = get(), b = get();
        cudaEventRecord(a, st);
        cudaError_t e = fn();
        cudaEventRecord(b, st);
        recs.push_back({cls, a, b});
        if (recs.size() > 4096) fold();  // bound the number of live events
        return e;
    }

    // Drop pending records and zero the sums (the caller synchronised).
    void reset(bool enable)
    {
        for (auto &r : recs) {
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
        for (int i = 0; i < IESH_K_COUNT; ++i) {
            ms[i] = 0.0;
            n[i] = 0;
        }
        on = enable;
    }

    void release()
    {
        for (auto &r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        recs.clear();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

// True for pageable or pinned host memory (a copy into it must be waited for).
inline bool is_host_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

}  // namespace iesh
