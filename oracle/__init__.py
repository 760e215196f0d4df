"""CPU oracle (test infrastructure only; see ``oracle/vibronic.py``)."""
