"""GB300-native D3Q27 cumulant LBM step on a block-refined mesh around an
L-system tree, with interpolated bounce-back and momentum-exchange drag.

The compute path is liblbm.so (CUDA for sm_103a) behind the C-ABI in
include/lbm.h; ``paper_2603_27954_gb300.lbm`` is its ctypes binding and
``paper_2603_27954_gb300.build`` compiles it.
"""
