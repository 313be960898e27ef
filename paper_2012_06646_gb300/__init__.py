"""GB300-native immersed-boundary spreading and interpolation (arXiv 2012.06646).

The compute path is the CUDA library libibgb.so (C ABI in include/ib.h),
built for sm_103a by `build.build()`.  This package is its thin Python
binding: `_abi` declares the C entry points under their C names, `plan`
wraps them for torch CUDA tensors, `autograd` makes spreading and
interpolation differentiable, and `serve` runs the continuous-batching
request loop over the batched entry points.  There is no CPU fallback.
"""

from .build import build  # noqa: F401


def load():
    """Load the CUDA library (raises if it has not been built)."""
    from . import _abi
    return _abi.load()


def __getattr__(name):
    if name in ("Plan", "Batch", "Stokes", "set_allocator", "use_torch_allocator"):
        from . import plan
        return getattr(plan, name)
    raise AttributeError(name)
