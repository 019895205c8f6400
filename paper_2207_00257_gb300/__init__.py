"""gbconv: dense 2D convolution for GB300 (sm_103a) behind a C ABI.

The convolution is the kernel at the centre of the PyTorch case of arXiv
2207.00257 (Sec. 1, Sec. 5.A-B). ``binding`` mirrors include/gbconv.h one to
one; ``functional`` adds torch-tensor conveniences and the autograd Function;
``synth`` draws the seeded synthetic inputs. The compiled library is built
in-tree by ``_build.build()``.
"""
from ._build import build  # noqa: F401
from . import binding  # noqa: F401

__all__ = ["build", "binding"]
