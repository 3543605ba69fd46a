/*
 * pccp_probe.h -- C ABI of libpccp_probe.so, the microbenchmarks that measure
 * the memory roofs bounding the propagation kernels on the current GPU.
 *
 * The method itself has no counterpart here: the paper's Sec. 5 names cache
 * use (shared memory per block) as the design driver of its GPU layout but
 * gives no roofline.  These probes measure the denominators of the library's
 * roofline fractions:
 *  - shared-memory load bandwidth (128 bytes per clock per SM nominal), the
 *    bound of propagation when table and stores are resident in shared memory;
 *  - the throughput of the relaxed CTA-scope shared atomics that carry every
 *    tell (the load/store semantics of Sec. 4);
 *  - L2 read bandwidth, the bound of the kernels that read a propagator table
 *    too large for shared memory from global memory.
 *
 * Conventions: 0 (PCCP_OK) on success, a negative PCCP_ERR_* code of pccp.h
 * otherwise.  Each call runs on the current device, allocates what it needs,
 * synchronises, and frees it before returning; `out` is a host pointer the
 * caller owns.
 */
#ifndef PCCP_PROBE_H
#define PCCP_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Probe kinds.  `work` in pccp_probe_result counts the unit named here. */
#define PCCP_PROBE_SMEM_LOAD 0 /* 16-byte shared loads, conflict-free: bytes */
#define PCCP_PROBE_SMEM_ATOM 1 /* atom.relaxed.cta.shared max.s32 on distinct
                                  words of each warp: operations */
#define PCCP_PROBE_SMEM_DOM 2  /* 8-byte relaxed interval loads (the kernels'
                                  form) at scattered indices: bytes */
#define PCCP_PROBE_L2_READ 3   /* 16-byte global loads cached in L2 only, over a
                                  32 MiB buffer already resident in L2: bytes */

typedef struct pccp_probe_result {
  double work;      /* units done by the timed launch */
  double ms;        /* its duration (CUDA events on the launching stream) */
  double sm_cycles; /* SM clock cycles the first CTA saw (clock64) */
  int n_sms;        /* multiprocessors of the device */
  int ctas;         /* CTAs launched */
} pccp_probe_result;

/* Runs probe `kind` once untimed and once timed.  iters <= 0 selects a
 * default that makes the timed launch last ~10-30 ms.  PCCP_ERR_INVALID for
 * an unknown kind or a NULL `out`. */
int pccp_probe(int kind, int iters, pccp_probe_result* out);

#ifdef __cplusplus
}
#endif

#endif /* PCCP_PROBE_H */
