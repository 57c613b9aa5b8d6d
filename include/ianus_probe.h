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
 *   kind 4: independent lop3.b32 and mad.wide.u32
 *           chains side by side (4 of each)         -> ops / clock / SM
 *   kind 5: mad.lo.u32 (32-bit multiply-add)        -> ops / clock / SM
 *   kind 6: three-input add (two add.u32)           -> ops / clock / SM
 *   kind 7: independent lop3.b32 and mad.lo.u32
 *           chains side by side (4 of each)         -> ops / clock / SM
 *   kind 8: mul.hi.u32 (32-bit high product)        -> ops / clock / SM
 *   kind 9: independent lop3.b32 and mul.hi.u32
 *           chains side by side (4 of each)         -> ops / clock / SM
 *   kind 10: Philox4x32-10 blocks with each product as a high and a low
 *           32-bit multiply                         -> blocks / clock / SM
 *   kind 11: Philox4x32-10 blocks with each product as a high multiply and
 *           a low multiply-add that cannot be merged into one 64-bit
 *           product                                 -> blocks / clock / SM
 *   kind 12: kind 3 plus 24 lop3.b32 of an independent chain per block
 *   kind 13: kind 11 plus the same 24 lop3.b32     -> blocks / clock / SM
 *   kind 14: as 13 with one product per round 64-bit, the other split
 * Kinds 4, 7 and 9 show whether the two instruction types issue in parallel
 * (about the sum of their separate rates) or share one issue slot.
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
