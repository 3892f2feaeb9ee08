"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package only *describes* circuits and noise models (which gate acts on which
qubit with which angle; which noise channel follows it). It holds none of the
method's arithmetic: no gate matrices, no Kraus matrices, no sampling.
"""
from .circuits import (  # noqa: F401
    OP_GATE, OP_NOISE, GATE, CHANNEL, Circuit, CircuitBuilder,
    brickwork, syndrome17, ansatz, uneven_batch, config, CONFIG_NAMES,
)
