// debug_checks.cuh -- index checks of a debug build (CR_DEBUG=1).
//
// A debug build checks every node, triangle and material index the traversal, shade and
// sum kernels use before it reads with it.  A failed check sets a bit of the scene's device
// error word and ends that ray (no out-of-bounds read); the host reports the word after the
// call.  In the normal build (CR_DEBUG=0) CR_DBG(...) expands to nothing.
#pragma once
#include <cuda_runtime.h>

#include "cr_internal.h"

namespace cr {

#ifndef CR_DEBUG
#define CR_DEBUG 0 // 1: a debug build that checks every node, triangle and material index it uses
#endif
#if CR_DEBUG
#define CR_DBG(...) __VA_ARGS__
#else
#define CR_DBG(...)
#endif
// error bits of the scene's device word in a debug build
constexpr uint32_t kDbgNode = 1u, kDbgTri = 2u, kDbgHit = 4u, kDbgMat = 8u;

// Debug builds: whether index idx < n; if not, the scene's error word gets `bit` (the caller
// then ends the ray instead of reading out of bounds).
__device__ __forceinline__ bool dbg_in_range(const SceneDev* sc, uint32_t idx, uint32_t bit, uint32_t n) {
    if (idx < n) return true;
    if (sc && sc->err) atomicOr(sc->err, bit);
    return false;
}


} // namespace cr
