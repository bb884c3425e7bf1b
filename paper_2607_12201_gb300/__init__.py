"""GB300-native Newton step of the Radau-collocation interior-point method.

``workloads`` draws seeded synthetic instances; ``collo`` is the thin ctypes
binding of the CUDA C-ABI library ``libcollo.so`` (built by ``build``).
"""
