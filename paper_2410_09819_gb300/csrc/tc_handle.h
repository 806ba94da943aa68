// Handle state and host helpers shared by the C-ABI translation units (internal).
#pragma once

#include "../../include/tile_chol.h"
#include "tc_internal.h"

#include <chrono>
#include <cstdio>
#include <string>
#include <vector>

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// One matrix of the current factorization (a single factor is a batch of one).
struct MatDesc {
    int64_t n = 0;
    int nt = 0;
    int64_t tile0 = 0;              // packed index of its tile (0, 0) in the concatenated W
    const double *A_dev = nullptr;  // the caller's matrix on the device (refinement)
    std::vector<uint8_t> map;       // nt x nt precision map (diagonal FP64)
    bool mixed = false;
};

struct tc_handle_s {
    tc_config cfg{};
    int device = 0;
    cudaStream_t s = nullptr;
    bool own_stream = false;
    std::string err;

    // last factorization
    int64_t n = 0;
    int b = 0, nt = 0;
    bool factored = false;
    bool mixed = false;
    double logdet = 0.0;
    double normA_inf = -1.0;
    std::vector<uint8_t> map;

    DevBuf W;          // FP64 factor tiles (the working copy of A)
    DevBuf Acopy;      // device copy of the caller's A when it was given in host memory
    const double *A_dev = nullptr;
    DevBuf status;     // int info word + padding
    DevBuf scratch;    // small doubles: logdet, norms, maxima
    DevBuf tables;     // schedule tables
    DevBuf partials;   // split-K partial blocks
    DevBuf vec;        // solve workspace
    DevBuf sumsq;      // tile sums of squares
    // mixed precision: operand pools, tables and tensor maps
    DevBuf pool_hi, pool_lo, pool16, pool8;
    DevBuf mxtab;
    CUtensorMap map_hi{}, map_lo{}, map16{}, map8{};
    // emulated FP64 updates: digit planes, their tables and tensor maps
    DevBuf dpool, ztab, invbuf;
    DevBuf stab;       // grouped batched-solve task tables
    CUtensorMap map_zx{}, map_zy{};
    tc::Z64Maps maps64{};                // 3D digit-plane maps of the mixed-precision update kernel
    // matrices of the last (batched) factorization
    std::vector<MatDesc> mats;
    std::vector<double> logdets;
    std::vector<int> infos;
    std::vector<double> normA_infs;
    // CUDA graph of the last batched factorization (replayed when the batch repeats)
    cudaGraphExec_t graph = nullptr;
    std::vector<int64_t> graph_key;
    uint64_t buf_gen = 0;        // bumped whenever a device buffer is (re)allocated
    uint64_t graph_gen = 0;      // buf_gen when the graph was captured (replay only if equal)
    DevBuf bstage;     // device copies of host-resident batch inputs
    // out-of-core: the factor lives in the caller's host matrix
    bool ooc = false;
    double *host_factor = nullptr;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    DevBuf logdiag;
    void *hcompact = nullptr;    // page-locked compact copies of final low-precision tiles
    size_t hcompact_bytes = 0;
    int64_t launches = 0;
    int64_t upd_launches[4] = {0, 0, 0, 0};
    unsigned long long *pairs_dev = nullptr;   // plane-pair counters of the mixed digit-plane updates
    unsigned long long pairs_exec[2] = {0, 0}; // their values after the last factorization

    // CUDA-event spans of the last factorization, by category (see Cat)
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    struct Span { int cat; cudaEvent_t a, b; };
    std::vector<Span> spans;
};

enum Cat { CAT_UPD64 = 0, CAT_UPD32, CAT_UPD16, CAT_UPD8, CAT_POTRF, CAT_TRSM, CAT_CONVERT, CAT_N };

namespace tc {

inline int set_err(tc_handle h, int code, const std::string &msg) {
    if (h) h->err = msg;
    return code;
}

inline int cuda_fail(tc_handle h, cudaError_t e, const char *what, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s) [tc_api.cu:%d]", what, cudaGetErrorName(e),
             cudaGetErrorString(e), line);
    return set_err(h, e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA, buf);
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call, __LINE__); \
    } while (0)

#define CK_LAUNCH()                                                                   \
    do {                                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, "kernel launch", __LINE__);    \
        ++h->launches;                                                                \
    } while (0)

inline bool on_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int ensure(tc_handle h, DevBuf &d, size_t bytes) {
    if (d.bytes >= bytes && d.p) return TC_OK;
    if (d.p) cudaFree(d.p);
    d.p = nullptr;
    d.bytes = 0;
    ++h->buf_gen;
    cudaError_t e = cudaMalloc(&d.p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return set_err(h, TC_ERR_OOM, buf);
    }
    d.bytes = bytes;
    return TC_OK;
}

inline void release(DevBuf &d) {
    if (d.p) cudaFree(d.p);
    d.p = nullptr;
    d.bytes = 0;
}

// Copy between any two pointers the runtime can classify (cudaMemcpyDefault).
inline int copy_any(tc_handle h, void *dst, const void *src, size_t bytes) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->s));
    return TC_OK;
}

inline cudaEvent_t next_event(tc_handle h) {
    if (h->events_used == h->events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->events.push_back(e);
    }
    return h->events[h->events_used++];
}

// Open a timed span on the handle's stream; close it with span_end.
inline int span_begin(tc_handle h, int cat) {
    cudaEvent_t a = next_event(h), b = next_event(h);
    if (!a || !b) return -1;
    cudaEventRecord(a, h->s);
    h->spans.push_back({cat, a, b});
    return (int)h->spans.size() - 1;
}

inline void span_end(tc_handle h, int id) {
    if (id >= 0) cudaEventRecord(h->spans[id].b, h->s);
}

// Sum the spans per category (the stream must be synchronised).
inline void span_totals(tc_handle h, double *ms) {
    for (int c = 0; c < CAT_N; ++c) ms[c] = 0.0;
    for (auto &sp : h->spans) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, sp.a, sp.b) == cudaSuccess) ms[sp.cat] += t;
        else cudaGetLastError();
    }
}

inline void spans_reset(tc_handle h) {
    h->spans.clear();
    h->events_used = 0;
}

inline double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

inline int check_nb(tc_handle h, int64_t n, int b) {
    if (!h) return TC_ERR_ARG;
    if (n < 1) return set_err(h, TC_ERR_ARG, "n must be >= 1");
    if (b < 64 || b > 4096 || b % 64) return set_err(h, TC_ERR_ARG, "tile size b must be a multiple of 64 in [64, 4096]");
    const int64_t nt = (n + b - 1) / b;
    if (nt > 65535) return set_err(h, TC_ERR_ARG, "too many tiles per column");
    return TC_OK;
}

int ooc_subst(tc_handle h, double *R, int64_t ldr, int nrhs, bool back, int64_t *h2d_bytes);

// Bound of the tensor-core kernels' pipeline waits for this handle (0: the kernels' default).
inline unsigned long long wait_limit_ns(tc_handle h) {
    return h->cfg.wait_limit_us > 0 ? (unsigned long long)h->cfg.wait_limit_us * 1000ull : 0ull;
}
// Failure-detection test hook (tc_config.wait_test): the tensor-core kernels first wait on a
// barrier that nothing arrives at.
inline int wait_test(tc_handle h) { return h->cfg.wait_test != 0; }

}  // namespace tc
