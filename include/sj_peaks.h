/*
 * sj_peaks.h -- instruction-rate microbenchmark exported by libsj.so.
 *
 * Not part of the join: the paper has no counterpart.  It measures the FP32
 * and FP64 FMA / add rates of the current device, which are the denominators
 * of the refinement kernels' arithmetic roofline (the join has no dense
 * contraction, so tensor-core peaks do not apply).
 */
#ifndef SJ_PEAKS_H
#define SJ_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t sms;              /* streaming multiprocessors                         */
    int32_t pad;
    double ffma_per_s;        /* FP32 fused multiply-adds per second (device-wide)  */
    double ffma_per_clk_sm;   /* ... per SM per SM clock cycle                      */
    double fadd_per_s;
    double fadd_per_clk_sm;
    double dfma_per_s;        /* FP64 fused multiply-adds per second                */
    double dfma_per_clk_sm;
    double dadd_per_s;
    double dadd_per_clk_sm;
} sj_peak_rates;

/* Runs four short kernels on the current device (a few milliseconds) and
 * fills *out.  Returns 0, -1 (NULL argument), -2 (allocation) or -4 (CUDA). */
int sj_peaks_measure(sj_peak_rates *out);

#ifdef __cplusplus
}
#endif

#endif /* SJ_PEAKS_H */
