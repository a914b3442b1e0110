/*
 * qap_peaks.h -- on-device microbenchmarks of libqapsa: the bandwidth, ALU
 * and synchronisation figures that bound the SA kernels on the current GPU.
 *
 * The paper (arXiv:1208.2675) has no counterpart; it times whole runs only
 * (section 4).  The Delta-matrix loop keeps its data on chip (registers, Tensor
 * Memory, shared memory) and waits on one CTA, cluster or grid barrier per
 * accepted swap, so the figures that bound it are the on-chip bandwidths, the
 * integer issue rates and the barrier latencies measured here, not HBM.
 *
 * qap_peaks_measure runs a fixed set of short kernels on the current device
 * (well under a second in total) and fills *out; it allocates a 64 MB scratch
 * buffer for the duration of the call.  Every figure comes from CUDA events
 * and clock64 counts of the kernels themselves; the SM clock used to convert
 * cycles to time is the one measured during the call.  Values that cannot be
 * measured on the device (a cluster size the device refuses) are 0.
 * Returns QAP_OK, QAP_E_INVAL (out == NULL), QAP_E_NOMEM or QAP_E_CUDA;
 * QAP_E_TIMEOUT if the grid barrier's bounded wait expired (it never should:
 * the grid is launched cooperatively, so all of its CTAs are resident).
 */
#ifndef QAP_PEAKS_H
#define QAP_PEAKS_H

#include <stdint.h>

#include "qap_sa.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qap_peaks {
  int32_t sm_count;               /* cudaDevAttrMultiProcessorCount            */
  int32_t smem_optin_bytes;       /* shared memory one CTA may opt in to       */
  int64_t l2_bytes;               /* cudaDevAttrL2CacheSize                    */
  double sm_mhz;                  /* SM clock during the kernels (cycles/time) */
  double smem_bytes_per_clk_sm;   /* volatile ld.shared.v4 streaming, one CTA per SM */
  double smem_gbs_chip;           /* the same over all SMs, GB/s               */
  double l2_gbs;                  /* ld.global.cg of an L2-resident 32 MB buffer, all SMs */
  double int32_ops_per_clk_sm;    /* independent 32-bit integer multiply-adds  */
  double dp4a_per_clk_sm;         /* independent dp4a (4 int8 products + add)  */
  double cta_barrier_ns;          /* __syncthreads, 640 threads                */
  double cluster_barrier_ns[5];   /* barrier.cluster at 2, 4, 8, 13, 16 CTAs   */
  double grid_barrier_ns;         /* release/acquire counter barrier, one CTA per SM */
  double l2_latency_ns;           /* one dependent ld.global.cg (L2 hit)       */
  double dsmem_latency_ns;        /* one dependent ld.shared::cluster of a peer CTA */
  double smem_latency_ns;         /* one dependent ld.shared                   */
  double l2_gbs_sm;               /* ld.global.cg of an L2-resident 8 MB buffer by
                                     one CTA of 1024 threads: what one SM draws  */
} qap_peaks;

QAP_EXPORT int qap_peaks_measure(qap_peaks *out);

#ifdef __cplusplus
}
#endif
#endif /* QAP_PEAKS_H */
