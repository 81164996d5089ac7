"""GB300 (sm_103a) implementation of the data-parallel hot path of the
critical-point-trajectory-preserving compressor for time-varying 2-D vector
fields.  The compute runs in the CUDA library built from ``csrc/``; the
``cpt`` module is its ctypes binding (argument marshalling only)."""
