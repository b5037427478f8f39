// Shared host/device utilities of libtdarisp (error handling, device buffers,
// kernel timing).  Internal header; the public interface is tdarisp.h.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "tdarisp.h"

namespace tr {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define TR_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw ::tr::Error(TR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TR_REQUIRE(cond, code, msg)                     \
    do {                                                \
        if (!(cond)) throw ::tr::Error((code), (msg));  \
    } while (0)

// Kernel launch bookkeeping: every launch goes through Prof::begin/end so the
// context can count launches and, when profiling is on, time each kernel
// with CUDA events on the launching stream.
// A few extra streams of a context for independent launches that are too small
// to fill the GPU one after another (fork from and join back to the context
// stream with events).
struct SideStreams {
    static constexpr int N = 4;
    cudaStream_t s[N] = {};
    cudaEvent_t fork = nullptr, join[N] = {};
    void ensure()
    {
        if (s[0]) return;
        for (int i = 0; i < N; ++i) {
            TR_CUDA(cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking));
            TR_CUDA(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
        }
        TR_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    }
    // side streams start after everything queued on st so far
    void begin(cudaStream_t st)
    {
        ensure();
        TR_CUDA(cudaEventRecord(fork, st));
        for (int i = 0; i < N; ++i) TR_CUDA(cudaStreamWaitEvent(s[i], fork, 0));
    }
    // st continues after everything queued on the side streams
    void end(cudaStream_t st)
    {
        for (int i = 0; i < N; ++i) {
            TR_CUDA(cudaEventRecord(join[i], s[i]));
            TR_CUDA(cudaStreamWaitEvent(st, join[i], 0));
        }
    }
    void release()
    {
        for (int i = 0; i < N; ++i) {
            if (s[i]) {
                cudaStreamSynchronize(s[i]);
                cudaStreamDestroy(s[i]);
            }
            if (join[i]) cudaEventDestroy(join[i]);
            s[i] = nullptr;
            join[i] = nullptr;
        }
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
    }
};

struct ProfRecord {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
};

struct Prof {
    bool enabled = false;
    long launches = 0;
    // bounded waits of the tensor-core pipelines launched through this recorder
    // (the context's tr_options.wait_cycles and wait_test): SM cycles before a
    // pipeline wait gives up (0: the kernels' default, about 1 s), and the test
    // switch under which the producer issues no operand loads
    long long wait_cycles = 0;
    int wait_stall = 0;
    std::vector<std::string> names;
    std::vector<ProfRecord> pending;
    std::vector<cudaEvent_t> pool;
    // accumulated per kind
    std::vector<long> n;
    std::vector<double> ms, fl, by;

    int kind(const char *name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.push_back(name);
        n.push_back(0);
        ms.push_back(0);
        fl.push_back(0);
        by.push_back(0);
        return (int)names.size() - 1;
    }
    cudaEvent_t ev() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        TR_CUDA(cudaEventCreate(&e));
        return e;
    }
    // NVTX ranges named after the kernel kind when TR_NVTX is set in the environment
    // (lets a profiler select one kind of kernel)
    int nvtx = -1;
    bool nvtx_on() {
        if (nvtx < 0) nvtx = std::getenv("TR_NVTX") ? 1 : 0;
        return nvtx == 1;
    }
    // returns a token to pass to end()
    int begin(cudaStream_t st, const char *name, double flops = 0, double bytes = 0) {
        launches += 1;
        if (nvtx_on()) nvtxRangePushA(name);
        if (!enabled) return -1;
        ProfRecord r;
        r.kind = kind(name);
        r.a = ev();
        r.b = ev();
        r.flops = flops;
        r.bytes = bytes;
        TR_CUDA(cudaEventRecord(r.a, st));
        pending.push_back(r);
        return (int)pending.size() - 1;
    }
    void end(cudaStream_t st, int tok) {
        if (tok >= 0) TR_CUDA(cudaEventRecord(pending[tok].b, st));
        if (nvtx_on()) nvtxRangePop();
    }
    // resolve pending events (synchronises on the last one)
    void flush() {
        for (auto &r : pending) {
            TR_CUDA(cudaEventSynchronize(r.b));
            float t = 0.f;
            TR_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            n[r.kind] += 1;
            ms[r.kind] += t;
            fl[r.kind] += r.flops;
            by[r.kind] += r.bytes;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    void reset() {
        flush();
        names.clear();
        n.clear();
        ms.clear();
        fl.clear();
        by.clear();
    }
    ~Prof() {
        for (auto &r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Error of the last launch, if any, as an exception naming the kernel kind
#define TR_CHECK_LAUNCH(what)                                                                        \
    do {                                                                                             \
        const cudaError_t ce_ = cudaGetLastError();                                                  \
        if (ce_ != cudaSuccess)                                                                      \
            throw ::tr::Error(TR_ECUDA, std::string("launch of ") + (what) + ": " + cudaGetErrorString(ce_)); \
    } while (0)

// Launch helper: checks the launch (an error names the kernel kind) and records it.
#define TR_LAUNCH(prof, stream, name, flops, bytes, ...)          \
    do {                                                          \
        int tok_ = (prof).begin((stream), (name), (flops), (bytes)); \
        __VA_ARGS__;                                              \
        const cudaError_t le_ = cudaGetLastError();               \
        if (le_ != cudaSuccess)                                   \
            throw ::tr::Error(TR_ECUDA, std::string("launch of ") + (name) + ": " + cudaGetErrorString(le_)); \
        (prof).end((stream), tok_);                               \
    } while (0)

// Device allocation accounting against a byte budget.
// Device blocks of a context kept for reuse by its later allocations of the
// same size instead of cudaFree, which waits for the whole device: builds of
// many contexts from several host threads (tr_build_batch) would otherwise
// serialise on each other's frees.  Blocks are taken only while `on` (the
// batched build: every use of a block is on the building context's streams,
// in order); they are freed when an allocation fails, beyond `cap` bytes, and
// with the context.  Pooled bytes do not count as used.
struct Pool {
    bool on = false;
    size_t cap = (size_t)1 << 30, held = 0;
    std::vector<std::pair<size_t, void *>> blocks;
    Pool() = default;
    Pool(const Pool &) = delete;
    Pool &operator=(const Pool &) = delete;
    ~Pool() { flush(); }
    void *take(size_t bytes)
    {
        for (size_t i = 0; i < blocks.size(); ++i)
            if (blocks[i].first == bytes) {
                void *q = blocks[i].second;
                blocks.erase(blocks.begin() + (long)i);
                held -= bytes;
                return q;
            }
        return nullptr;
    }
    bool put(void *q, size_t bytes)
    {
        if (!on || held + bytes > cap) return false;
        blocks.emplace_back(bytes, q);
        held += bytes;
        return true;
    }
    bool flush()
    {
        const bool any = !blocks.empty();
        for (auto &b : blocks) cudaFree(b.second);
        blocks.clear();
        held = 0;
        return any;
    }
};

struct Budget {
    size_t limit = 0, used = 0, peak = 0;
    Pool pool;
};

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    Budget *budget = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (!budget || !budget->pool.put(p, n * sizeof(T))) cudaFree(p);
            if (budget) budget->used -= n * sizeof(T);
        }
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, Budget *b, const char *what) {
        if (count == n && p) return;
        release();
        if (count == 0) return;
        size_t bytes = count * sizeof(T);
        if (b && b->limit && b->used + bytes > b->limit)
            throw Error(TR_ENOMEM, std::string("device budget exceeded allocating ") + what);
        void *q = b && b->pool.on ? b->pool.take(bytes) : nullptr;
        cudaError_t e = cudaSuccess;
        if (q) {
            p = (T *)q;
        } else {
            e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess && b && b->pool.flush()) {  // blocks kept for reuse go back first
                cudaGetLastError();
                e = cudaMalloc(&p, bytes);
            }
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            throw Error(TR_ENOMEM, std::string("cudaMalloc failed for ") + what + ": " +
                                       cudaGetErrorString(e));
        }
        n = count;
        budget = b;
        if (b) {
            b->used += bytes;
            if (b->used > b->peak) b->peak = b->used;
        }
    }
    // grow-only allocation for scratch space
    void reserve(size_t count, Budget *b, const char *what) {
        if (count <= n && p) return;
        alloc(count, b, what);
    }
};

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace tr
