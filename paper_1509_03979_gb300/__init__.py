"""GB300 (sm_103a) greedy compressive-sensing decoders with CG-based weighted least squares.

The compute path is the CUDA library libcs_gb300.so (csrc/); `binding` marshals PyTorch
tensors into its C ABI (include/cs_gb300.h).  `synth` generates seeded synthetic inputs.
Submodules are imported explicitly (`from paper_1509_03979_gb300 import binding`).
"""
