// Per-rank kernel tables (the run-time -> compile-time rank dispatch of Algorithm 7, as a
// plain table of instantiations indexed by the effective rank).
#pragma once

namespace triot {
// row kernels: op ROW_EMBED / ROW_CROP by element size (2, 4, 8 bytes), ROW_PRODUCT by
// dtype; nouter = effective rank - 1 in [0, 23]
const void* embed_kernel_ptr(int es, int nouter);
const void* crop_kernel_ptr(int es, int nouter);
const void* product_kernel_ptr(int dtype, int nouter);
// moment kernels by dtype and effective rank D in [1, 24]
const void* moment_kernel_ptr(int dtype, int D);
const void* combine_kernel_ptr();
}  // namespace triot
