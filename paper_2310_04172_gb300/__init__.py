"""GB300 (sm_103a) library for the 6D MCL particle sensor update in TSDF maps.

The computation lives in ``libmcl.so`` behind the C ABI of ``include/mcl.h``;
``paper_2310_04172_gb300.mcl`` is its thin Python binding (same names).
"""
from . import mcl  # noqa: F401
from ._build import build  # noqa: F401
