"""GB300-native (sm_103a) Monte Carlo sample-average estimation of the
mean-variance objective, its gradient and the Frank-Wolfe loop of
arXiv 2404.11631 (Sec. 3.1, Eqs. 3-5, Algorithm 1).

The compute path is the C-ABI library ``libsaa.so`` (hand-written CUDA);
``paper_2404_11631_gb300.saa`` is its thin ctypes binding and
``paper_2404_11631_gb300.autograd`` the ``torch.autograd.Function`` on top.
Submodules load lazily so that ``inputs`` can be used without a GPU.
"""
import importlib

__all__ = ["saa", "autograd", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
