"""GraphGuess (arXiv 2104.10039) hot path for GB300: CUDA kernels behind the
C ABI of include/gg.h (libgg.so), with a ctypes binding in ``gg``.

``from paper_2104_10039_gb300 import gg`` loads libgg.so and raises if it has
not been built; ``build.build()`` compiles it (nvcc, sm_103a). ``metrics``
holds the accuracy metrics of Sec. 4.2 (host-side evaluation helpers).
"""
