"""GB300-native multi-hit weighted set cover with P-DFS (libmh).

The compute path is the CUDA library ``libmh.so`` (sources in ``csrc/``, C ABI
in ``include/mh.h``); ``mh`` is its thin ctypes binding.
"""
from . import mh  # noqa: F401
from .mh import (Handle, MHError, MHLibraryError, Result, mh_create, mh_create_device, mh_destroy,  # noqa: F401
                 mh_handle_info, mh_last_error, mh_set_stream, mh_solve, mh_solve_ex)
