"""GB300-native instant colorization of Gaussian splats (arXiv 2604.17155).

The compute path is the C-ABI library libicgs.so (hand-written sm_103a CUDA, declared in
include/icgs.h); `paper_2604_17155_gb300.icgs` is its thin Python binding.
"""
