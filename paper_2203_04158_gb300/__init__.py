"""GB300 (sm_103a) ranking, on-the-fly H·v and Lanczos for quantum many-body
states, after Wallerberger & Held, "Trie-based ranking of quantum many-body
states" (arXiv:2203.04158).

The compute path is the C-ABI library ``libgbrank.so`` (``include/gbrank.h``);
``gbrank`` is its thin binding.  Build it with :func:`build.build`.
"""
from . import gbrank  # noqa: F401
from .gbrank import *  # noqa: F401,F403
