/*
 * sbli_probe.h -- arithmetic-throughput probe of the current GPU, the
 * denominator of the ALU roofline that the stage kernels are reported
 * against (binary64 is bound by GB300's FP64 pipe, not by HBM).
 *
 * The paper has no counterpart: it reports the nominal peak of each machine
 * (Table 2).  Here the peak is measured on the machine that runs the stages.
 * Conventions (status codes, sbli_last_error) are those of sbli.h.
 */
#ifndef SBLI_PROBE_H
#define SBLI_PROBE_H

#include "sbli.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Fused multiply-add throughput of the current device in one precision.
 *   precision  SBLI_FP64 (binary64 FMA) or SBLI_FP32 (binary32 FMA);
 *   iters      loop trips per thread, >= 1; each trip advances 8 independent
 *              FMA chains by 2 steps (16 FMAs); the launch fills every SM to
 *              full occupancy (on GB300 in binary64 about 8 us per trip);
 *   sink_dev   8 bytes of device memory the kernel may write (it keeps the
 *              chains live; in practice it is never written);
 *   stream     cudaStream_t (NULL = legacy default stream);
 *   flop_per_s out: 2 * FMAs executed / kernel time (CUDA events on stream);
 *   ms         out (may be NULL): the kernel time in milliseconds.
 * Synchronises the stream.  SBLI_EINVAL for another precision, iters < 1 or
 * null pointers; SBLI_ECUDA if a launch or event call fails. */
SBLI_API int sbli_probe_fma_rate(int precision, long long iters, double* sink_dev, void* stream, double* flop_per_s,
                                 float* ms);

#ifdef __cplusplus
}
#endif
#endif /* SBLI_PROBE_H */
