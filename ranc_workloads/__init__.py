"""Seeded synthetic workloads (networks and inputs) shared by the CUDA path,
the CPU oracle, the tests and the benchmark.  Holds no simulation arithmetic."""

from .nets import (DEST_DTYPE, KIND_CORE, KIND_NONE, KIND_OUTPUT, NEG_RESET, NEG_SATURATE, Net,
                   make_net, mnist_512core, pack_bits_lsb, random_net, layered_net, rate_coded_inputs, tiny_5core,
                   empty_dest, truenorth_ref)
from . import rng

__all__ = ["DEST_DTYPE", "KIND_CORE", "KIND_NONE", "KIND_OUTPUT", "NEG_RESET", "NEG_SATURATE", "Net",
           "make_net", "mnist_512core", "pack_bits_lsb", "random_net", "layered_net", "rate_coded_inputs", "tiny_5core",
           "empty_dest", "truenorth_ref", "rng"]
