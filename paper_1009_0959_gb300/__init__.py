"""GB300-native vector order-statistic filters (VMF, BVDF, AMNFE/G, EVMF)
with exact and minimax elementary functions (arXiv 1009.0959).

  paper_1009_0959_gb300.vfilt   binding of the C ABI (include/vfilt.h)
  paper_1009_0959_gb300.build   in-tree nvcc build of libvfilt.so (sm_103a)
  paper_1009_0959_gb300.synth   seeded synthetic inputs (images, noise)

The binding is imported lazily so that the input generator can be used on a
machine without the CUDA library; any filter call without it raises.
"""


def __getattr__(name):
    if name in ("vfilt", "build", "synth"):
        import importlib
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
