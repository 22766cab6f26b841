"""Balanced butterfly counting on GB300 (placeholder; binding added below)."""
