// Many independent cells at once on a pool of streams: each cell's host-driven solver runs on
// one of up to OF_POOL_STREAMS internal streams, one host thread per stream, so that the
// kernels of different cells overlap on the GPU.  Used by the batched entry points.
#pragma once

#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "of_internal.cuh"

namespace of {

constexpr int OF_POOL_STREAMS = 8;

// Runs body(c) for every cell c with grids[c]->stream switched to a worker stream.  The
// workers first wait for the work already queued on the cells' shared stream; the shared
// stream then waits for every worker, and is synchronised before the call returns.  body
// returns a status (and may throw Error); the first failing cell's status is returned with
// its message.  The grids must all use the same stream and device and must not be touched
// by other threads meanwhile.
template <class Body>
of_status run_on_stream_pool(int ncells, of_grid* const* grids, Body&& body) {
    of_grid* g0 = grids[0];
    const cudaStream_t shared = g0->stream;
    const int T = std::min(ncells, OF_POOL_STREAMS);
    std::vector<cudaStream_t> wstream(T, nullptr);
    std::vector<cudaEvent_t> wdone(T, nullptr);
    cudaEvent_t start = nullptr;
    std::vector<of_status> status(ncells, OF_OK);
    std::vector<std::string> message(ncells);
    auto cleanup = [&]() {
        for (int t = 0; t < T; ++t) {
            if (wstream[t]) cudaStreamDestroy(wstream[t]);
            if (wdone[t]) cudaEventDestroy(wdone[t]);
        }
        if (start) cudaEventDestroy(start);
    };
    try {
        OF_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
        note_resource();
        OF_CUDA(cudaEventRecord(start, shared));
        for (int t = 0; t < T; ++t) {
            OF_CUDA(cudaStreamCreateWithFlags(&wstream[t], cudaStreamNonBlocking));
            OF_CUDA(cudaEventCreateWithFlags(&wdone[t], cudaEventDisableTiming));
            note_resource();
            note_resource();
            OF_CUDA(cudaStreamWaitEvent(wstream[t], start, 0));
        }
    } catch (const Error& e) {
        cleanup();
        return e.code;
    }
    auto work = [&](int t) {
        cudaSetDevice(g0->device);
        for (int c = t; c < ncells; c += T) {
            of_grid* g = grids[c];
            g->stream = wstream[t];
            try {
                status[c] = body(c);
            } catch (const Error& e) {
                status[c] = e.code;
            } catch (...) {
                status[c] = OF_ECUDA;
            }
            if (status[c] != OF_OK) message[c] = of_last_error();
            g->stream = shared;
        }
        cudaEventRecord(wdone[t], wstream[t]);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < T; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
    of_status worst = OF_OK;
    try {
        for (int t = 0; t < T; ++t) OF_CUDA(cudaStreamWaitEvent(shared, wdone[t], 0));
        OF_CUDA(cudaStreamSynchronize(shared));
    } catch (const Error& e) {
        worst = e.code;
    }
    cleanup();
    for (int c = 0; c < ncells && worst == OF_OK; ++c)
        if (status[c] != OF_OK) {
            worst = status[c];
            set_error("cell %d: %s", c, message[c].c_str());
        }
    return worst;
}

}  // namespace of
