"""CPU oracle for the TRIOT hot path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The library under paper_1608_00099_gb300/ never imports it.
"""
