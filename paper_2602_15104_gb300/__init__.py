"""GB300 (sm_103a) library for the data-parallel hot path of the ABCMB linear
Einstein-Boltzmann method (arXiv 2602.15104): batched perturbation ODEs ->
CMB sources -> line-of-sight projection -> C_ell^{TT,TE,EE}.

The compute path is the CUDA library libabcmb.so (C ABI in include/abcmb.h);
`paper_2602_15104_gb300.abcmb` is its thin Python binding.
"""
