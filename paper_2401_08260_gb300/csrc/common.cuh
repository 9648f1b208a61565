// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "slk.h"

namespace slk {

// NFFT window taps of FP32 plans as polynomials: degree (the even/odd split of the kernels
// assumes 8), and the widest window (cells)
constexpr int kWinPolyDeg = 8;
constexpr int kWinPolyMaxM = 16;

// ---------------------------------------------------------------- errors

struct Error {
    slk_status status;
    std::string msg;
};

void set_last_error(const std::string& msg);

[[noreturn]] void fail(slk_status st, const char* fmt, ...);

#define SLK_CHECK_CUDA(call)                                                                      \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            ::slk::fail(e_ == cudaErrorMemoryAllocation ? SLK_ERR_OOM : SLK_ERR_CUDA, "%s:%d %s: %s", \
                        __FILE__, __LINE__, #call, cudaGetErrorString(e_));                       \
    } while (0)

#define SLK_CHECK_LAUNCH() SLK_CHECK_CUDA(cudaGetLastError())

#define SLK_REQUIRE(cond, ...)                                  \
    do {                                                        \
        if (!(cond)) ::slk::fail(SLK_ERR_INVALID, __VA_ARGS__); \
    } while (0)

// ---------------------------------------------------------------- memory

// Stream-ordered device allocation from the device's default memory pool.
void* dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);

// Owning device buffer (freed stream-ordered on the stream it was allocated on
// unless moved).
template <class T>
struct DevBuf {
    T* ptr = nullptr;
    size_t count = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t st) { alloc(n, st); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { *this = static_cast<DevBuf&&>(o); }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            reset();
            ptr = o.ptr;
            count = o.count;
            stream = o.stream;
            o.ptr = nullptr;
            o.count = 0;
        }
        return *this;
    }
    ~DevBuf() { reset(); }
    void alloc(size_t n, cudaStream_t st) {
        reset();
        stream = st;
        count = n;
        ptr = n ? static_cast<T*>(dev_alloc(n * sizeof(T), st)) : nullptr;
    }
    void reset() {
        if (ptr) dev_free(ptr, stream);
        ptr = nullptr;
        count = 0;
    }
    size_t bytes() const { return count * sizeof(T); }
    T* get() const { return ptr; }
};

// Memory kind of a user pointer.
bool is_device_pointer(const void* p);

// ---------------------------------------------------------------- kernel timing

// Brackets one kernel launch: counts it and, while timing is enabled, records
// CUDA events around it on its stream (see slk_timing_*).
class LaunchScope {
   public:
    LaunchScope(const char* name, cudaStream_t st);
    ~LaunchScope();
    LaunchScope(const LaunchScope&) = delete;
    LaunchScope& operator=(const LaunchScope&) = delete;

   private:
    const char* name_;
    cudaStream_t st_;
    cudaEvent_t start_ = nullptr;
};

#define SLK_CAT2(a, b) a##b
#define SLK_CAT(a, b) SLK_CAT2(a, b)
#define SLK_TIMED(name, st) ::slk::LaunchScope SLK_CAT(slk_scope_, __LINE__)(name, st)

// ---------------------------------------------------------------- device helpers

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <class T>
struct Cplx {
    T re, im;
};

__device__ inline void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ inline void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }

// Order-preserving map of an FP32 / FP64 key to an unsigned integer.
__device__ inline uint32_t key_bits(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline unsigned long long key_bits(double f) {
    unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(f));
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

}  // namespace slk
