// Bounds checks of the debug build (compiled with -DGFK_DEBUG; the release
// build compiles every check to `true`).
//
// The library registers each device buffer it allocates (and, for the
// allocation-free entry point, the caller's buffers) in a table of address
// ranges in device memory.  In the debug build the kernels check every state,
// trajectory, checkpoint, record and series access against that table before
// making it: an access that does not lie wholly inside one registered range
// sets a bit of a status word, records the first such address, and is skipped
// (a load yields zeros).  Nothing traps, so the context stays usable and the
// host reads the word with gfk_debug_status.
#pragma once

#include <cstddef>

#if defined(__CUDACC__)
#define GFK_HD __host__ __device__
#else
#define GFK_HD
#endif

namespace gfk {

// Status bits (gfk_debug_status): which kind of access failed its check.
enum : unsigned {
    kDbgState = 1u,        // a walker's state planes (positions, log-weight, sign)
    kDbgRecord = 2u,       // a block's per-move record
    kDbgSeries = 4u,       // a per-step series row or an exported walker
    kDbgPositions = 8u,    // the gradient's checkpoints, segment or trajectory
    kDbgTableFull = 16u,   // more live buffers than table entries: checks were off
};

constexpr int kDbgRanges = 256;

// Host registry of device buffers (gfk_debug.cu; no-ops in the release build):
// register [p, p + bytes) after an allocation, unregister p before its free.
void debug_register(const void* p, size_t bytes);
void debug_unregister(const void* p);

// 1 if the bytes [p, p + bytes) lie inside one of the n half-open ranges
// [lo[k], hi[k]).  An empty access (bytes 0) must still start inside a range.
GFK_HD inline bool dbg_in_ranges(const unsigned long long* lo, const unsigned long long* hi,
                                 int n, unsigned long long p, unsigned long long bytes) {
    for (int k = 0; k < n; ++k)
        if (p >= lo[k] && p < hi[k] && bytes <= hi[k] - p) return true;
    return false;
}

}  // namespace gfk

#if defined(GFK_DEBUG) && defined(__CUDACC__)
namespace gfk {

// The registered ranges (n < 0: the table overflowed and checks are off).
struct DbgTable {
    unsigned long long lo[kDbgRanges], hi[kDbgRanges];
    int n;
};
extern __device__ DbgTable g_dbg_table;
extern __device__ unsigned g_dbg_flags;
extern __device__ unsigned long long g_dbg_addr;

__device__ __forceinline__ bool dbg_ok(const void* p, unsigned long long bytes, unsigned code) {
    const int n = g_dbg_table.n;
    if (n < 0) return true;
    const unsigned long long a = (unsigned long long)p;
    if (dbg_in_ranges(g_dbg_table.lo, g_dbg_table.hi, n, a, bytes)) return true;
    atomicOr(&g_dbg_flags, code);
    atomicCAS(&g_dbg_addr, 0ull, a);
    return false;
}

}  // namespace gfk
#define GFK_DBG_OK(p, bytes, code) ::gfk::dbg_ok((p), (bytes), (code))
#else
#define GFK_DBG_OK(p, bytes, code) true
#endif
