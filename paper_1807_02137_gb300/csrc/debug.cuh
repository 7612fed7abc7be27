// debug.cuh -- index bounds checks of the MG_DEBUG build.
//
// Built with -DMG_DEBUG, every global-memory access of the solver's kernels that goes through
// MG_DBG_OK is first compared with the size of the buffer it addresses (for a grid function of
// a level: n x pitch elements; for the member masks: 2 n npm and 2 m npn words).  An index out
// of range does not fault: the access is skipped (a load gives 0) and the kernel records the
// event in a device error word of its translation unit:
//   word[0]  bit s set: site s saw an out-of-range index (sites: DebugSite below)
//   word[1]  the first out-of-range index seen, word[2] its site + 1, word[3] the count.
// The host reads and clears the words of every translation unit through mg_debug_status.  No
// check traps or asserts.  In the default build MG_DBG_OK is the constant true and no code is
// generated for it.
#pragma once

#include <cuda_runtime.h>

namespace segmg {

// MG_DEBUG builds: each translation unit registers the reader of its device error words at load
// time; mg_debug_status ORs them together.  Returns the number of readers so far.
int register_debug_reader(int (*read)(unsigned long long *words, int clear));

enum DebugSite : int {
    kDbgSetup = 0,       // image set-up, initial phi, fitting fields, restriction of data
    kDbgHaloLoad,        // the 36 x 36 and 32 x 32 tile loads of the snapshot and residual
    kDbgSnapshot,        // snapshot stores (f, G, class) and weight loads
    kDbgMaskStore,       // member masks written by the snapshot
    kDbgMaskLoad,        // member masks read by the sweeps
    kDbgSweep,           // sweep tile loads and stores (non-TMA accesses)
    kDbgResidual,        // residual, restriction, FAS right-hand side
    kDbgInterp,          // interpolation and correction
    kDbgBottom,          // one-block and cluster bottom of the V-cycle
    kDbgCoarse,          // coarsest-grid solve
    kDbgOther,           // line smoothers, AOS, learned weights
    kDbgSites
};

#ifdef MG_DEBUG
// One set of words per translation unit (no relocatable device code is needed).
static __device__ unsigned long long g_dbg_word[4];

__device__ __noinline__ static void dbg_report(long long idx, int site) {
    atomicOr(&g_dbg_word[0], 1ull << site);
    if (atomicCAS(&g_dbg_word[2], 0ull, (unsigned long long)(site + 1)) == 0ull)
        g_dbg_word[1] = (unsigned long long)idx;
    atomicAdd(&g_dbg_word[3], 1ull);
}

__device__ __forceinline__ bool dbg_ok(long long idx, long long lim, int site) {
    if ((unsigned long long)idx < (unsigned long long)lim) return true;
    dbg_report(idx, site);
    return false;
}

// Host side: copies (and optionally clears) this translation unit's words.
static int dbg_read_words(unsigned long long *out, int clear) {
    if (cudaMemcpyFromSymbol(out, g_dbg_word, sizeof(g_dbg_word)) != cudaSuccess) return -1;
    if (clear) {
        const unsigned long long z[4] = {0, 0, 0, 0};
        if (cudaMemcpyToSymbol(g_dbg_word, z, sizeof(z)) != cudaSuccess) return -1;
    }
    return 0;
}
static const int g_dbg_registered = register_debug_reader(&dbg_read_words);

#define MG_DBG_OK(idx, lim, site) ::segmg::dbg_ok((long long)(idx), (long long)(lim), (site))
#else
#define MG_DBG_OK(idx, lim, site) true
#endif

// Checked element load and store: p[i] with i < lim in the debug build; the plain access in the
// default build.
template <typename T>
__device__ __forceinline__ T ldc(const T *p, size_t i, size_t lim, int site) {
#ifdef MG_DEBUG
    if (!dbg_ok((long long)i, (long long)lim, site)) return T();
#else
    (void)lim; (void)site;
#endif
    return p[i];
}
template <typename T>
__device__ __forceinline__ void stc(T *p, size_t i, size_t lim, int site, T v) {
#ifdef MG_DEBUG
    if (!dbg_ok((long long)i, (long long)lim, site)) return;
#else
    (void)lim; (void)site;
#endif
    p[i] = v;
}

}  // namespace segmg
