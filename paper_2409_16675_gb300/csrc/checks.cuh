// checks.cuh -- device-side bounds checks of the debug build (-DHE_CHECKS).
//
// Every global load and store of the kernels goes through the macros below.
// In the normal build they are the plain accesses.  In the checks build each
// access tests its address range against a sorted table of the device
// allocations the library may touch (its own allocations, registered when
// made, and the allocations holding the caller's buffers of every call).  A
// miss is counted in a device error word that records the first bad address
// and source line; the access is skipped (a load yields zero, a store does
// nothing, an object check makes the thread return) and nothing traps.  The
// checked entry points (checks.cpp) read the word back after each call and
// return HE_ERR_INVALID_ARG.
//
// Without relocatable device code every translation unit has its own copy of
// the table and the error word; HE_CHECKS_UNIT(name) defines the host
// functions that fill and read them.
#pragma once
#include <cstdint>

#ifdef HE_CHECKS
namespace he {
constexpr int kCheckRanges = 4096;
struct CheckTable {
    int n;                           // ranges in use, sorted by lo, disjoint
    int pad_;
    unsigned long long lo[kCheckRanges], hi[kCheckRanges];  // [lo, hi)
};
struct CheckError {
    unsigned int count;              // violations since the last read
    unsigned int line;               // source line of the first
    unsigned long long addr;         // its address
};
static __device__ CheckTable g_check_table;
static __device__ CheckError g_check_error;

// true when [p, p + bytes) lies inside one registered range
static __device__ __noinline__ bool check_span(const void *p, unsigned long long bytes, int line) {
    const unsigned long long a = (unsigned long long)p;
    int lo = 0, hi = g_check_table.n - 1, found = -1;
    while (lo <= hi) {                   // last range whose start is <= a
        const int mid = (lo + hi) >> 1;
        if (g_check_table.lo[mid] <= a) { found = mid; lo = mid + 1; }
        else hi = mid - 1;
    }
    if (found >= 0 && a + bytes <= g_check_table.hi[found]) return true;
    if (atomicAdd(&g_check_error.count, 1u) == 0) {
        g_check_error.line = (unsigned)line;
        g_check_error.addr = a;
    }
    return false;
}
}  // namespace he

template <class T>
__device__ __forceinline__ T he_ld_(const T *p, int line) {
    return he::check_span(p, sizeof(T), line) ? *p : T{};
}
template <class T>
__device__ __forceinline__ T he_ldg_(const T *p, int line) {
    return he::check_span(p, sizeof(T), line) ? __ldg(p) : T{};
}
template <class T>
__device__ __forceinline__ T he_ldca_(const T *p, int line) {
    return he::check_span(p, sizeof(T), line) ? __ldca(p) : T{};
}
template <class T, class V>
__device__ __forceinline__ void he_st_(T *p, const V &v, int line) {
    if (he::check_span(p, sizeof(T), line)) *p = v;
}
#define HE_LD(p) he_ld_((p), __LINE__)
#define HE_LDG(p) he_ldg_((p), __LINE__)
#define HE_LDCA(p) he_ldca_((p), __LINE__)
#define HE_ST(p, v) he_st_((p), (v), __LINE__)
// a whole object (a table entry read through a reference): false if outside
#define HE_OBJ_OK(p) he::check_span((p), sizeof(*(p)), __LINE__)
// n consecutive objects starting at p
#define HE_SPAN_OK(p, n) he::check_span((p), sizeof(*(p)) * (unsigned long long)(n), __LINE__)

#define HE_CHECKS_UNIT(name)                                                                       \
    int checks_put_##name(const he::CheckTable *t) {                                               \
        return cudaMemcpyToSymbol(he::g_check_table, t, sizeof(he::CheckTable)) == cudaSuccess ? 0 : -1; \
    }                                                                                              \
    int checks_take_##name(he::CheckError *e) {                                                    \
        static const he::CheckError zero = {0, 0, 0};                                              \
        if (cudaMemcpyFromSymbol(e, he::g_check_error, sizeof *e) != cudaSuccess) return -1;       \
        return cudaMemcpyToSymbol(he::g_check_error, &zero, sizeof zero) == cudaSuccess ? 0 : -1;  \
    }
#else
#define HE_LD(p) (*(p))
#define HE_LDG(p) __ldg(p)
#define HE_LDCA(p) __ldca(p)
#define HE_ST(p, v) (*(p) = (v))
#define HE_OBJ_OK(p) true
#define HE_SPAN_OK(p, n) true
#define HE_CHECKS_UNIT(name)
#endif
