"""GB300-native QEM E-step (arXiv 2503.08264): massively parallel importance
weighting over plated hierarchical models, in hand-written sm_103a kernels
behind the C ABI of include/qem.h.

``synth`` (seeded workloads) imports without CUDA; ``qem`` (the binding) loads
libqem.so and needs torch with a CUDA device.
"""
__all__ = ["synth", "qem", "build"]
