"""GB300 three-site TEBD: C-ABI library (libptebd.so, hand-written sm_103a kernels)
and its thin Python binding.  See include/ptebd.h for the ABI."""
from .binding import SuperSiteTEBD, TEBD, TEBDError, batch_step, gate_host, gate_host_supersite, load  # noqa: F401
