"""GB300-native FFT-PIM apply (arXiv 2312.02376).

The compute path is libpim.so (CUDA, sm_103a) behind the C ABI in
include/pim.h; `paper_2312_02376_gb300.pim` is its Python binding and
`paper_2312_02376_gb300.inputs` the seeded synthetic workloads.
"""
