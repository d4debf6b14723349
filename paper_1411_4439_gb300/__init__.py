"""GB300-native multi-right-hand-side HISQ Dslash and conjugate gradient.

The compute path is the CUDA library lib/libhisq.so (C ABI in include/hisq.h);
``paper_1411_4439_gb300.hisq`` is its Python binding with the same names.
Build the library with ``paper_1411_4439_gb300.build_lib.build()``.
"""
from . import hisq  # noqa: F401
from .hisq import (  # noqa: F401
    HISQ_AOS, HISQ_BUNDLE, HISQ_F16, HISQ_F32, HISQ_F64, HISQ_MAP_L2_PREFETCH, HISQ_MAP_PACKED,
    HISQ_MAP_COMPACT, HISQ_MAP_TILE_XY, HISQ_MAP_PIPELINED, HISQ_MAP_PIPELINED2, HISQ_MAP_STAGED, HISQ_OP_D2M_DMU2, HISQ_OP_D3M_DMU3, HISQ_OP_D4M_DMU4, HISQ_OP_DM_DMU,
    HISQ_OP_M, HISQ_OP_MDAG, HISQ_R12, HISQ_R14, HISQ_R18, HISQ_SOA, Gauge, HisqError,
    cg_params, hisq_apply_m, hisq_cdot, hisq_cdot_noalloc, hisq_cg_default_params,
    hisq_cg_solve, hisq_cg_solve_batched, hisq_autotune_bundle, hisq_autotune_dslash, hisq_bundle_pack, hisq_bundle_unpack, hisq_dslash, hisq_dslash_ex, hisq_gauge_free, hisq_gauge_info,
    hisq_gauge_load, hisq_gauge_load_tuned, hisq_get_dslash_mapping, hisq_get_dslash_mapping_ex, hisq_link_compress, hisq_link_force,
    hisq_link_reconstruct, hisq_mdagm, hisq_set_dslash_mapping, hisq_version,
)

__all__ = [n for n in dir() if n.startswith(("hisq_", "HISQ_"))] + ["Gauge", "HisqError", "cg_params"]
