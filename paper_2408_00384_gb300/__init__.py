"""GB300-native stabilizer-tableau simulator (Aaronson-Gottesman formalism, the
Clifford backend of arXiv:2408.00384, section "Simulation of Clifford circuits").

The compute path is libtab.so (CUDA, sm_103a) behind the C ABI in include/tab.h;
``paper_2408_00384_gb300.tab`` is its ctypes binding.  Importing the binding
fails loudly when the library has not been built: there is no CPU fallback.
"""

__all__ = ["tab"]
