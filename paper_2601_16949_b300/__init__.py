"""B300-native RT-TDA propagation: the sigma build H(t)c inside an RK4 stepper.

Importing the package is cheap; the CUDA library is loaded when the binding
is first used (``paper_2601_16949_b300.binding``), and that import fails
loudly if the library has not been built.
"""

__all__ = ["binding", "synth", "build"]


def __getattr__(name):
    if name in ("binding", "synth", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
