/*
 * qcams_debug.h - test-support entry points of the GB300 QCT library.
 *
 * These are not part of the trajectory path: they expose pieces of the
 * integrator's arithmetic and of the library's bookkeeping so that tests can
 * check them in isolation.  They are exported by the same shared library as
 * the entry points of qcams.h and follow its conventions (atomic units,
 * caller-owned memory, status codes, asynchronous on `cuda_stream` unless
 * stated).
 */
#ifndef QCAMS_DEBUG_H
#define QCAMS_DEBUG_H

#include <stdint.h>

#include "qcams.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Diagnostic (test support): evaluates, for n device arguments x[i], the
 * integrator's table-driven exponential (Tang's method, used for the Morse
 * and Buckingham exponentials) into out_table[i] and CUDA's exp into
 * out_cuda[i] (device arrays).  Asynchronous.
 */
int qcams_debug_exp(const double* x, double* out_table, double* out_cuda, int64_t n,
                    void* cuda_stream);

/*
 * Diagnostic (test support): the elementary functions of the integrator's
 * Morse force law (Sec. 3.2 item 1, V = De (1 - e^{-alpha (r - re)})^2 - De)
 * on n device squared distances s[i]:
 *   out_rinv[i] = 1/sqrt(s[i])   (FP32 hardware estimate refined in FP64;
 *                                 NaN outside 2^-126 <= s < 2^128),
 *   out_arg[i]  = x = alpha_re - alpha r,  r = s[i] out_rinv[i],
 *   out_exp[i]  = e^x            (table method with the index rounded in FP32).
 * alpha > 0, 0 < alpha_re < 700, else QCAMS_E_INVALID.  Device arrays of
 * length n, caller-owned.  Asynchronous.
 */
int qcams_debug_force_math(const double* s, double alpha, double alpha_re, double* out_rinv,
                           double* out_arg, double* out_exp, int64_t n, void* cuda_stream);

/*
 * Diagnostic (test support): the integrator's float-float dot product, the
 * arithmetic of its stage corrections and embedded error estimate (the
 * Dormand-Prince step of Sec. 3.2): for n rows i,
 *   out[i]   = sum_{q<m} w[q] a[i*m + q]  as a double (both operands split
 *              into float pairs, compensated accumulation, rebuilt on the
 *              integer pipe),
 *   out_f[i] = the same sum rounded to FP32.
 * a: device [n][m] row-major; w: device [m]; 1 <= m <= 8, else
 * QCAMS_E_INVALID.  Device outputs of length n, caller-owned.  Asynchronous.
 */
int qcams_debug_ff_dot(const double* a, const double* w, int32_t m, double* out, float* out_f,
                       int64_t n, void* cuda_stream);

/*
 * Whether the per-device context of the current device exists: *out = 1 if
 * a call that uses it (qcams_levels, qcams_init_states, qcams_run_batch,
 * qcams_analyze, qcams_autotune, qcams_last_run_stats) has created it since
 * the last qcams_shutdown, else 0.  Host-only and synchronous; it creates
 * nothing, allocates nothing and enqueues no work.
 */
int qcams_debug_context_exists(int32_t* out);

#ifdef __cplusplus
}
#endif

#endif /* QCAMS_DEBUG_H */
