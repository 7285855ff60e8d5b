"""CPU oracle for the data-mapping analysis hot path.

TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded reference written
from the paper (Algorithms 1-5 of Sec. 5 and the Sec. 7.6 estimate) and from
the FP128 v1 hash definition.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the GPU library never does.

The compiled part lives in ``odp_oracle.cpp``; :func:`build` compiles it with
g++ into ``liboracle.so`` next to this file.
"""

from .oracle import (  # noqa: F401
    build,
    lib,
    fp128,
    fp128_many,
    analyze,
    analyze_bruteforce,
    FINDING_DTYPE,
    SITE_DTYPE,
    SUMMARY_FIELDS,
    OracleResult,
)
