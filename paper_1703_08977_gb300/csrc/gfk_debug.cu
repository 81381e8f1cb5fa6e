// Host side of the debug build's bounds checks (gfk_debug.h): the table of
// registered device buffers and gfk_debug_status.  In the release build the
// registry calls do nothing and gfk_debug_status reports a release build.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include "gfk.h"
#include "gfk_debug.h"

#ifdef GFK_DEBUG
namespace gfk {

__device__ DbgTable g_dbg_table;
__device__ unsigned g_dbg_flags;
__device__ unsigned long long g_dbg_addr;

namespace {

std::mutex g_mu;
std::vector<std::pair<unsigned long long, unsigned long long>> g_ranges;   // [lo, hi)
bool g_full = false;

// Copies the host table to the current device (callers hold g_mu).
void push_table() {
    static DbgTable t;
    t.n = g_full ? -1 : (int)g_ranges.size();
    for (size_t k = 0; k < g_ranges.size() && k < (size_t)kDbgRanges; ++k) {
        t.lo[k] = g_ranges[k].first;
        t.hi[k] = g_ranges[k].second;
    }
    cudaMemcpyToSymbol(g_dbg_table, &t, sizeof(t));
    // in place before any later launch, on whichever stream
    cudaDeviceSynchronize();
}

}  // namespace

void debug_register(const void* p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long lo = (unsigned long long)p, hi = lo + bytes;
    for (auto& r : g_ranges)
        if (r.first == lo) {
            r.second = r.second > hi ? r.second : hi;
            push_table();
            return;
        }
    if (g_ranges.size() >= (size_t)kDbgRanges) g_full = true;
    else g_ranges.emplace_back(lo, hi);
    push_table();
}

void debug_unregister(const void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_mu);
    // kernels still running may use the buffer: let them finish first
    cudaDeviceSynchronize();
    const unsigned long long lo = (unsigned long long)p;
    for (size_t k = 0; k < g_ranges.size(); ++k)
        if (g_ranges[k].first == lo) {
            g_ranges.erase(g_ranges.begin() + (long)k);
            break;
        }
    push_table();
}

}  // namespace gfk

extern "C" gfk_status gfk_debug_status(int32_t* debug_build, uint32_t* flags, uint64_t* first_addr,
                                       int32_t clear) {
    if (debug_build) *debug_build = 1;
    unsigned f = 0;
    unsigned long long a = 0;
    if (cudaMemcpyFromSymbol(&f, gfk::g_dbg_flags, sizeof(f)) != cudaSuccess ||
        cudaMemcpyFromSymbol(&a, gfk::g_dbg_addr, sizeof(a)) != cudaSuccess) {
        (void)cudaGetLastError();
        return GFK_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lock(gfk::g_mu);
        if (gfk::g_full) f |= gfk::kDbgTableFull;
    }
    if (flags) *flags = f;
    if (first_addr) *first_addr = a;
    if (clear) {
        const unsigned zf = 0;
        const unsigned long long za = 0;
        if (cudaMemcpyToSymbol(gfk::g_dbg_flags, &zf, sizeof(zf)) != cudaSuccess ||
            cudaMemcpyToSymbol(gfk::g_dbg_addr, &za, sizeof(za)) != cudaSuccess) {
            (void)cudaGetLastError();
            return GFK_ECUDA;
        }
    }
    return GFK_OK;
}

#else

namespace gfk {
void debug_register(const void*, size_t) {}
void debug_unregister(const void*) {}
}  // namespace gfk

extern "C" gfk_status gfk_debug_status(int32_t* debug_build, uint32_t* flags, uint64_t* first_addr,
                                       int32_t) {
    if (debug_build) *debug_build = 0;
    if (flags) *flags = 0;
    if (first_addr) *first_addr = 0;
    return GFK_OK;
}

#endif
