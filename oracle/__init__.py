"""Plain FP64 CPU oracle for the hybrid thermal pseudopotential LB boiling step.

This package is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import it. The
product path (``paper_1501_03857_gb300``) never imports, links or executes it.
"""

from .lbm import *  # noqa: F401,F403
from .wetting import cap_density, contact_angle_cap  # noqa: F401
