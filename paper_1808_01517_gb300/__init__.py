"""GB300-native (sm_103a) DELIMIT spherical layers: Signal2SH, SH2Signal and the
local spherical convolution (Koppers & Merhof, arXiv:1808.01517).

The compute lives in ``libdelimit.so`` (C ABI: ``include/delimit.h``); this
package holds the build script, the ctypes binding (``_lib``), the torch
layers (``layers``) and the seeded synthetic inputs (``synth``).  Importing
the package does not load the library; ``layers`` and ``_lib.get()`` do.
"""

__all__ = ["synth", "layers", "build"]
