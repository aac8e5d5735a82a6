"""python -m paper_2210_13641_gb300.probe: the ceilings for the hash-grid traffic."""

from . import main

main()
