"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This package produces inputs only -- buffer contents and event logs shaped
like the paper's workloads -- and holds none of the analysed method's
arithmetic (no hashing, no pattern detection).  Every generator is
deterministic in its seed.  Random numbers come from SplitMix64 (Steele, Lea,
Flood 2014) used as a counter-based generator, implemented once in numpy
(:mod:`synth.prng`) and once as a CUDA fill kernel (``gen.cu``).
"""

from . import prng, content, traces  # noqa: F401
