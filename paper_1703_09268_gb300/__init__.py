"""GB300-native frequency-domain FWI misfit and adjoint-state gradient.

Submodules are imported lazily so that input generation (`synth`) works on
machines without the CUDA library:
  synth     seeded synthetic workloads (no method arithmetic)
  helm      ctypes binding of the C ABI in libhelm.so (include/helm.h)
  autograd  torch.autograd.Function around misfit_and_gradient
"""
__all__ = ["synth", "helm", "autograd"]
