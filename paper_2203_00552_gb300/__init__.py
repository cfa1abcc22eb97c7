"""GB300-native ddLPB energy and analytical forces (arXiv:2203.00552).

The compute path is the sm_103a CUDA library libddlpb.so (C ABI in
include/ddlpb.h); this package builds it (build.py), binds it (_binding.py)
and draws seeded synthetic solutes (synth.py).
"""
from ._binding import (DDLPB_FP64, DDLPB_MIXED, OP_AB, OP_AB_F16, OP_ABT, OP_ABT_F16, OP_C, OP_CT, OP_FP32, OP_L,
                       OP_LT, Context, DDLPBError, default_options, library)

__all__ = ["Context", "DDLPBError", "library", "default_options", "DDLPB_FP64", "DDLPB_MIXED", "OP_L", "OP_LT",
           "OP_AB", "OP_ABT", "OP_C", "OP_CT", "OP_FP32", "OP_AB_F16", "OP_ABT_F16"]
