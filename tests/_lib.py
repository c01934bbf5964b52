"""Build libtfi in-tree if it is stale, then import the binding."""
from paper_2609_34025_b300 import build as _build

_build.build()

import paper_2609_34025_b300 as tfi  # noqa: E402,F401
