"""GB300-native (sm_103a) differentiable tile-based Gaussian rasterizer with the
entropy term on blending weights and the periodic scale reset of
"Speeding Up the Learning of 3D Gaussians with Much Shorter Gaussian Lists"
(arXiv 2603.09277).

Submodules are imported lazily so that the seeded input generators
(``scenes``) can be used without the CUDA library:

- ``scenes``: seeded synthetic inputs (no rasterizer arithmetic).
- ``gs``: ctypes binding of the C-ABI library ``libgs.so`` (fails loudly if
  the library has not been built).
- ``rasterize``: torch.autograd.Function wrappers over the C-ABI.
- ``build``: compiles ``csrc/*.cu`` into ``libgs.so`` for sm_103a.
- ``schedule``: the resolution scheduler and the epoch plan of the scale
  reset and the entropy term (host logic).
"""
import importlib

__all__ = ["scenes", "gs", "rasterize", "build", "schedule"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
