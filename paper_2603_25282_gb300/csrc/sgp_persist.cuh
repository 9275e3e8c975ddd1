// sgp_persist.cuh -- the persistent work-queue kernel of 2D ensembles.
//
// An ensemble of independent runs on grids of different sizes advances a
// chunk of steps in ONE launch: every CTA repeatedly takes the next work
// item from a device queue, an item being one CTA-sized tile of one pass
// (an x-pass or a y-line pass of Sec. 3's splitting) of one member.  The
// queue lists the items pass by pass (all members' tiles of pass 0, then
// of pass 1, ...).  A member's pass may start only when all tiles of its
// previous passes are done: a per-member counter of finished tiles orders
// them.  A CTA waits only for items that precede its own in the queue,
// which running CTAs have already taken, so the waits always end; each
// wait is nevertheless bounded (a number of clock64 cycles), after which
// the kernel records the failure in a control word, every CTA stops, and
// the host reports SGP_ETIMEOUT.
#pragma once
#include "sgp_launch.cuh"

namespace sgp {

enum { PK_XPASS = 0, PK_LINE = 1 };

// One pass of one grid group; the program lists them pass by pass, the
// groups in order inside a pass (entry p * groups + g).
template <typename R>
struct PersistPass {
  int kind;             // PK_XPASS or PK_LINE (lines along y)
  int N;                // line length of the pass
  int tiles;            // work items per member
  int members;          // members of the group
  XPassArgs<R> x;       // arguments of an x-pass (kind PK_XPASS)
  LPassArgs<R> l;       // arguments of a line pass (kind PK_LINE)
};

// Shape of a program (kernel parameter): passes alternate x-pass, line
// pass, x-pass, ... (2D), every x-pass has IX work items and every line
// pass IL; inside a pass the groups' items follow each other.  A work item
// is up to kTilesPerItem consecutive tiles of one member.
constexpr int kPersistMaxGroups = 32;
constexpr int kTilesPerItem = 2;
struct PersistLayout {
  int IX, IL;                            // work items of an x-pass and of a line pass
  int groups;
  int xoff[kPersistMaxGroups + 1];       // items of the groups before g in an x-pass
  int loff[kPersistMaxGroups + 1];       // the same in a line pass
  int xt[kPersistMaxGroups];             // tiles per member of an x-pass
  int lt[kPersistMaxGroups];             // tiles per member of a line pass
  int xi[kPersistMaxGroups];             // items per member of an x-pass
  int li[kPersistMaxGroups];             // items per member of a line pass
  int base[kPersistMaxGroups];           // the group's first member (completion counter)
};

// Control block of a launch (device memory).
struct PersistCtl {
  unsigned long long head;   // next work item; reset before every launch
  long long withhold;        // test hook: this item does not signal completion (-1: none)
  int err;                   // 0, or 1 after a bounded wait gave up (kept until the host clears it)
  int pad;
  long long err_item;        // the item whose wait gave up
};

// Line lengths the persistent kernel is compiled for (both pass geometries
// have 256 threads per CTA for them).
bool persist_supported(int N);
// Geometry of the persistent kernel's passes: x-pass rows per CTA and
// line-pass columns per CTA for line length N.
template <typename R> int persist_xrows(int N);
template <typename R> int persist_ltile(int N);
// Set the kernel's shared-memory attribute on the current device and return
// the CTAs that fit on one SM.
template <typename R> cudaError_t persist_prepare(int* blocks_per_sm);
template <typename R>
cudaError_t launch_persistent(const PersistPass<R>* prog, const PersistLayout& lay, int nitems,
                              int* done, PersistCtl* ctl, long long wait_cycles, int grid,
                              cudaStream_t s);

}  // namespace sgp
