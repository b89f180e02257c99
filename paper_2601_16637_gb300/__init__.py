"""GB300-native selected-basis diagonalization (SBD) for SQD workflows.

The compute path is the CUDA library libsbd.so (C ABI in include/sbd.h);
`binding` marshals Python arguments to it, `workloads` draws seeded synthetic
inputs and `build` compiles the library in-tree.  Importing the package loads
nothing; `binding.load()` loads the library and fails loudly if it is absent.
"""
__all__ = ["binding", "build", "workloads"]
