// Per-rank kernel tables (the run-time -> compile-time rank dispatch of Algorithm 7, as a
// plain table of instantiations indexed by the effective rank).
#pragma once

namespace triot {
// row kernels: op ROW_EMBED / ROW_CROP by element size (2, 4, 8 bytes), ROW_PRODUCT by
// dtype; nouter = effective rank - 1 in [0, 23]
const void* embed_kernel_ptr(int es, int nouter);
// embed into a view whose written rows are not back to back (strided A)
const void* embed_view_kernel_ptr(int es, int nouter);
const void* crop_kernel_ptr(int es, int nouter);
const void* product_kernel_ptr(int dtype, int nouter);
// moment kernels by dtype and effective rank D in [1, 24]; m > 0 selects the block-column
// kernel (f32/bf16/f16 only) with D - m outer axes
// m > 0: block-column kernel for blocks of B elements (the last m axes)
const void* moment_kernel_ptr(int dtype, int D, int m = 0, int B = 0);
const void* moment_blk32_kernel_ptr(int dtype, int B);
const void* moment_wb_kernel_ptr(int dtype, int B);
const void* moment_blk64_kernel_ptr(int B, int DO);
// sticky flags of the block moment kernels (a bounded wait gave up); reading clears them
void b64_read_device_flag(int* flag);
void b32_read_device_flag(int* flag);
void wb_read_device_flag(int* flag);
const void* combine_kernel_ptr();
// f64 moment by marginals (rows x columns split)
const void* moment_mx64_kernel_ptr();
// float storage by marginals: V = elements per vector load (1: single-element loads)
const void* moment_mx32_kernel_ptr(int dtype, int V);
// moment of a product of tensors: one kernel per dtype and tensor count (1..4)
const void* moment_prod_kernel_ptr(int dtype, int ntensors);
// the same on rows shorter than kMPRowsMaxL elements (CTA tiles of rows, mprod_rows.h)
const void* moment_prod_rows_kernel_ptr(int dtype, int ntensors);
}  // namespace triot
