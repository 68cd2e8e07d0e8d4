"""GB300-native fast level set evolutions (arXiv 1409.7474).

The compute path is the CUDA library ``liblse.so`` (built in-tree from
``csrc/``) behind the C ABI declared in ``include/lse.h``; ``lse`` is its thin
ctypes binding.  ``scenes`` draws seeded synthetic inputs.  Importing this
package loads nothing; ``paper_1409_7474_gb300.lse`` loads the library and
raises if it has not been built.
"""
__version__ = "0.1.0"
