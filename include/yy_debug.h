/*
 * yy_debug.h - test hooks of libyy (not needed by applications).
 *
 * Fault injection is done on the host only: these hooks make the library's
 * own allocation wrapper report failure so the error paths can be exercised
 * without touching the GPU's state.
 */
#ifndef YY_DEBUG_H
#define YY_DEBUG_H

#ifdef __cplusplus
extern "C" {
#endif

/* Make the n-th following device allocation made by the library fail with
 * YY_ERR_OOM (n = 0: the next one).  A negative n disables the hook.  Not
 * thread-safe; process-wide. */
void yy_debug_fail_alloc_after(int n);

#ifdef __cplusplus
}
#endif

#endif /* YY_DEBUG_H */
