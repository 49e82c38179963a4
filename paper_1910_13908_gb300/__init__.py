"""SAGE/EM direction-dependent calibration on one GB300: the CUDA library
(csrc/, C ABI in include/sagecal_gb.h), its ctypes binding (sagecal), the
synthetic inputs (synth) and the calibration server (serve)."""
import os as _os

# Jobs calibrated at once run on separate CUDA streams.  The device takes
# their launches through a fixed number of hardware work queues, 8 unless
# the process asks for more before its CUDA context exists; streams that
# share a queue wait on each other's launches.  32 is the most a process
# can have.  A value set by the user is kept.
_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
