// Shared internal definitions of the HSIM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/hsim.h"

namespace hsim {

// Errors travel as exceptions inside the library and become a status plus a
// thread-local message at the ABI boundary.
struct Error : std::runtime_error {
    hsim_status status;
    Error(hsim_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] inline void fail(hsim_status s, const std::string &msg) { throw Error(s, msg); }

// Records the message that hsim_last_error() returns on this thread.
void set_last_error(const std::string &msg);

#define HSIM_CHECK_ARG(cond, msg)                                  \
    do {                                                           \
        if (!(cond)) ::hsim::fail(HSIM_E_INVALID_ARG, (msg));      \
    } while (0)

#define HSIM_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            ::hsim::fail(HSIM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                          " (" __FILE__ ":" + std::to_string(__LINE__) + ")"); \
    } while (0)

// Every kernel launch goes through this so that launches are counted and
// launch errors are caught at the call site.
extern std::atomic<uint64_t> g_launches;
#define HSIM_LAUNCHED()                                                                   \
    do {                                                                                  \
        ::hsim::g_launches.fetch_add(1, std::memory_order_relaxed);                        \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            ::hsim::fail(HSIM_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_) + \
                                          " (" __FILE__ ":" + std::to_string(__LINE__) + ")"); \
    } while (0)

// Raise a kernel's dynamic shared-memory limit once per device to the largest
// size any of its launches uses.  The limit is an attribute of the function
// on the current device shared by all host threads: setting it per launch to
// that launch's size races with launches of the same kernel from other
// threads (batched solves).
constexpr int kMaxDevices = 64;
#define HSIM_SMEM_LIMIT_ONCE(func, max_bytes)                                                        \
    do {                                                                                              \
        static std::once_flag once_[::hsim::kMaxDevices];                                             \
        static cudaError_t err_[::hsim::kMaxDevices] = {};                                            \
        int dev_ = 0;                                                                                 \
        HSIM_CUDA(cudaGetDevice(&dev_));                                                              \
        if (dev_ < 0 || dev_ >= ::hsim::kMaxDevices) ::hsim::fail(HSIM_E_CUDA, "device index above 63"); \
        std::call_once(once_[dev_], [&] {                                                             \
            err_[dev_] = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(max_bytes)); \
        });                                                                                           \
        HSIM_CUDA(err_[dev_]);                                                                        \
    } while (0)

// Owning device buffer.
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            fail(HSIM_E_NOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                                   " bytes failed: " + cudaGetErrorString(e));
        }
        n = count;
    }
    // grow-only reallocation (contents not kept)
    void reserve(size_t count) { if (count > n) alloc(count); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void upload(const std::vector<T> &h, cudaStream_t s) {
        alloc(h.size());
        if (!h.empty()) HSIM_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    std::vector<T> download(cudaStream_t s) const {
        std::vector<T> h(n);
        if (n) HSIM_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        return h;
    }
};

// Host CSR pattern (+ optional values).
struct Csr {
    int n_rows = 0, n_cols = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

struct DevCsr {
    int n_rows = 0, n_cols = 0;
    int64_t nnz = 0;
    DevBuf<int> ptr, col;
    void upload(const Csr &c, cudaStream_t s) {
        n_rows = c.n_rows;
        n_cols = c.n_cols;
        nnz = c.nnz();
        ptr.upload(c.ptr, s);
        col.upload(c.col, s);
    }
};

}  // namespace hsim
