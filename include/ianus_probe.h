/*
 * ianus_probe.h -- C ABI of libianus_probe.so, the integer-throughput probe
 * that supplies the roofline denominator of the sweep kernels.
 *
 * The paper has no counterpart: its update engines are FPGA logic whose
 * throughput is fixed by the clock and the number of update cells
 * (Sec. 3.1, Sec. 4.1.1).  On the GPU the sweep is bound by 32-bit integer
 * issue (Philox multiplies and three-input logic), while the usual measured
 * peaks (a memory copy, a bf16 GEMM) say nothing about integer issue, so
 * this probe measures per-SM integer rates directly.
 *
 * ianus_probe_int(kind, blocks_per_sm, out):
 *   kind 0: lop3.b32 (three-input logic)           -> ops / clock / SM
 *   kind 1: mad.wide.u32 (32x32+64 multiply-add)    -> ops / clock / SM
 *   kind 2: one mad.wide.u32 and two lop3.b32 per
 *           step (the Philox round mix)             -> ops / clock / SM
 *   kind 3: Philox4x32-10 blocks                    -> blocks / clock / SM
 * Each block of 256 threads runs independent dependency chains and times
 * itself with the SM cycle counter; *out receives the median over blocks of
 * (ops per block / cycles) times blocks_per_sm.  Runs on the current device
 * and synchronises it.  Returns 0 on success, 1 for bad arguments, 3 for a
 * CUDA error.
 */
#ifndef IANUS_PROBE_H
#define IANUS_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

int ianus_probe_int(int kind, int blocks_per_sm, double* out);

#ifdef __cplusplus
}
#endif

#endif
