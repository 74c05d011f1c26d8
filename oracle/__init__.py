"""FP64 CPU oracle of OCSC -- test infrastructure only (see ``oracle/ocsc.py``)."""
from .ocsc import *  # noqa: F401,F403
from . import ocsc  # noqa: F401
