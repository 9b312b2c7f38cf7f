"""CPU oracle (test infrastructure only; see ``oracle/cp.py``)."""
