"""GB300 (sm_103a) implementation of the TRIOT hot path (Heyl & Serang, arXiv 1608.00099).

The compute lives in libtriot.so (hand-written CUDA kernels behind the C ABI declared in
include/triot.h); `paper_1608_00099_gb300.triot` is its ctypes binding.  Importing the
package does not load the library: the first operation does, and fails loudly if the
library has not been built (`paper_1608_00099_gb300.build.build()`).
"""
from .triot import (BATCH_FUSED, BATCH_PHASED, EMBED_NOPAD, OP_CROP, OP_EMBED, OP_MOMENT,  # noqa: F401
                    OP_PRODUCT, BatchPlan, TriotError, lib, triot_autotune, triot_canonicalize,
                    triot_crop, triot_device_status, triot_embed, triot_fastdiv_check, triot_moment,
                    triot_moment_workspace_size, triot_product, triot_tune_clear, triot_tune_get,
                    triot_tune_load, triot_tune_save, triot_tune_set, version)
