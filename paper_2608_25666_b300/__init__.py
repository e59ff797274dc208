"""PRISM QP projection on one B300: C-ABI library libprism_proj + thin binding.

Import ``paper_2608_25666_b300.prism_proj`` for the binding (it loads the
compiled CUDA library on first use) and ``paper_2608_25666_b300.workloads`` for
the seeded synthetic inputs.
"""
