"""GB300-native multilevel CPCP solver (arXiv 2206.13369 hot path).

The CUDA library lives in ``_lib/libcpcp.so`` (built by ``build.build()``);
``cpcp`` is its Python binding and ``workloads`` the seeded synthetic inputs.
"""
