"""Code generator for the pointwise algebra of the CUDA kernels.

``python -m paper_2606_02053_gb300.codegen.generate`` rewrites
``paper_2606_02053_gb300/csrc/generated/*.cuh``; the generated files are
committed, and a test checks that they are up to date.
"""
