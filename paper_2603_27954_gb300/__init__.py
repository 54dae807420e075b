"""GB300-native D3Q27 cumulant LBM step on a block-refined mesh around an
L-system tree, with interpolated bounce-back and momentum-exchange drag.

The compute path is liblbm.so (CUDA for sm_103a) behind the C-ABI in
include/lbm.h; ``lbm`` is its ctypes binding.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def build(force=False):
    from . import build as _b
    return _b.build(force=force)
