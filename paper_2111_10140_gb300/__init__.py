"""GB300-native ANOVA-Gaussian fast summation and kernel ridge regression.

The compute path is the C-ABI library ``libanova_gb300.so`` built from
``csrc/`` (hand-written CUDA for sm_103a); ``binding`` marshals arguments to
it.  Importing this package does not load the library; ``binding.lib()`` does,
and raises if it is missing.
"""
__all__ = ["binding", "workloads"]
