"""GB300-native batched rigid/articulated physics step (CUDA, sm_103a) behind a C ABI.

    from paper_2106_14405_gb300 import Sim
    sim = Sim(scenegen.make_batch(2), scenegen.params_for(2))
    sim.step(4)

The engine is the shared library built from csrc/ (see include/sim.h); there is
no Python or CPU implementation of it, and loading fails loudly without it.
"""
from . import build  # noqa: F401  (module: build.build() compiles libsim.so)
from ._native import SimError, load  # noqa: F401
from .engine import Sim  # noqa: F401
