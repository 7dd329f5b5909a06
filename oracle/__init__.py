"""CPU oracle for the chemistry hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library.
"""
